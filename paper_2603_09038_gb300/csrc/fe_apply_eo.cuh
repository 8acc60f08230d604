// Even-odd phases of the fused apply (policies with kEvenOdd, tables TabEO): FP64, FP32, and the
// compensated float-float policy of the high orders.
//
// GB300's FP64 pipe (2 DFMA per clock per SM) bounds the FP64 apply, and FP32 issue bounds the
// float-float one, so the lever is the number of arithmetic instructions.  The 1D tables of
// Eq. (2) are symmetric under reversal of both indices (B[Q-1-q][D-1-d] = B[q][d],
// G[Q-1-q][D-1-d] = -G[q][d]; GLL nodes and Gauss points are symmetric about the element centre),
// so every line contraction out = M u is done on the even and odd parts of u by two half-size
// products whose sum and difference give the outputs in mirrored pairs (TabEO documents the
// formulas).  For a line of D inputs and Q outputs this costs about QD/2 + D + Q operations
// instead of QD; the x and y phases share one split of a line between the B and G contractions,
// and the z phase pairs the quadrature points qz and Q-1-qz so that the transposed contraction
// takes the even and odd parts of the pointwise products directly.
//
// The phases are written once over an element-operations policy (EoOps): plain arithmetic for
// FP64 and FP32, and for float-float pairs the compensated products of the direct scheme
// (exact product, FMA-corrected cross terms) with TwoSum-based additions for the splits and
// the joins, every output normalised as in the direct scheme.  Each function is one phase of
// pa_apply_block with the generic phase's shared-memory layout, inputs and outputs; only the
// contraction arithmetic differs (and with it the rounding, within the same parity bar).
#pragma once

#include "fe_arith.cuh"

namespace fe {
namespace eo {

// ---- element operations
template <class R>
struct EoOps {  // FP64 / FP32
  using T = R;
  static __device__ __forceinline__ T add(T a, T b) { return a + b; }
  static __device__ __forceinline__ T sub(T a, T b) { return a - b; }
  static __device__ __forceinline__ T mul(T c, T u) { return c * u; }
  static __device__ __forceinline__ T mac(T c, T u, T acc) { return fma(c, u, acc); }
  static __device__ __forceinline__ T fin(T a) { return a; }
};

template <>
struct EoOps<f2> {  // float-float, compensated
  using T = f2;
  // a + b, unnormalised: TwoSum of the high words, the low words added to its error
  static __device__ __forceinline__ T add(T a, T b) {
    const f2 s = two_sum(a.h, b.h);
    return f2{s.h, f_add(s.l, f_add(a.l, b.l))};
  }
  static __device__ __forceinline__ T sub(T a, T b) { return add(a, f2{-b.h, -b.l}); }
  // c u: the exact product of the high words plus the FMA-accumulated cross terms
  static __device__ __forceinline__ T mul(T c, T u) {
    const float p = f_mul(c.h, u.h);
    float e = f_fma(c.h, u.h, -p);
    e = f_fma(c.h, u.l, e);
    e = f_fma(c.l, u.h, e);
    return f2{p, e};
  }
  static __device__ __forceinline__ T mac(T c, T u, T acc) {
    f2_mad(acc, c.h, c.l, u);
    return acc;
  }
  static __device__ __forceinline__ T fin(T a) { return f2_norm(a); }
};

// ---- host: the tables B, G [Q][D] (G may be null: zero) and their even-odd halves, formed in
//      long double and rounded once to the element type (float pairs: high word and remainder)
template <class R>
inline R eo_round(long double v) {
  return (R)v;
}
template <>
inline f2 eo_round<f2>(long double v) {
  const float h = (float)v;
  return f2{h, (float)(v - (long double)h)};
}

template <class R, int D, int Q>
inline void fill(const double* B, const double* G, TabEO<R, D, Q>* t) {
  using L = long double;
  using TT = TabEO<R, D, Q>;
  auto Bq = [&](int q, int d) { return (L)B[q * D + d]; };
  auto Gq = [&](int q, int d) { return G ? (L)G[q * D + d] : (L)0; };
  for (int q = 0; q < Q; ++q)
    for (int d = 0; d < D; ++d) {
      t->B[q * D + d] = eo_round<R>(Bq(q, d));
      t->G[q * D + d] = eo_round<R>(Gq(q, d));
    }
  for (int o = 0; o < TT::QE; ++o) {
    for (int i = 0; i < TT::DE; ++i) t->bS[o][i] = eo_round<R>((Bq(o, i) + Bq(Q - 1 - o, i)) / 2);
    for (int i = 0; i < TT::DH; ++i) t->gS[o][i] = eo_round<R>((Gq(o, i) + Gq(Q - 1 - o, i)) / 2);
  }
  for (int o = 0; o < TT::QH; ++o) {
    for (int i = 0; i < TT::DH; ++i) t->bD[o][i] = eo_round<R>((Bq(o, i) - Bq(Q - 1 - o, i)) / 2);
    for (int i = 0; i < TT::DE; ++i) t->gD[o][i] = eo_round<R>((Gq(o, i) - Gq(Q - 1 - o, i)) / 2);
  }
  for (int k = 0; k < TT::DE; ++k) {
    for (int q = 0; q < TT::QE; ++q) t->btS[k][q] = eo_round<R>((Bq(q, k) + Bq(q, D - 1 - k)) / 2);
    for (int q = 0; q < TT::QH; ++q) t->gtS[k][q] = eo_round<R>((Gq(q, k) + Gq(q, D - 1 - k)) / 2);
  }
  for (int k = 0; k < TT::DH; ++k) {
    for (int q = 0; q < TT::QH; ++q) t->btD[k][q] = eo_round<R>((Bq(q, k) - Bq(q, D - 1 - k)) / 2);
    for (int q = 0; q < TT::QE; ++q) t->gtD[k][q] = eo_round<R>((Gq(q, k) - Gq(q, D - 1 - k)) / 2);
  }
}

// ---- primitives
// ue[i] = v[i] + v[N-1-i], uo[i] = v[i] - v[N-1-i] (i < N/2); ue takes the middle entry of an
// odd line
template <int N, class R>
__device__ __forceinline__ void split(const R (&v)[N], R (&ue)[(N + 1) / 2], R (&uo)[N / 2]) {
  using O = EoOps<R>;
#pragma unroll
  for (int i = 0; i < N / 2; ++i) {
    ue[i] = O::add(v[i], v[N - 1 - i]);
    uo[i] = O::sub(v[i], v[N - 1 - i]);
  }
  if constexpr (N % 2 == 1) ue[N / 2] = v[N / 2];
}

// out[o] = S[o] + Dd[o], out[N-1-o] = S[o] - Dd[o]; the middle output of an odd line is S
template <int N, class R>
__device__ __forceinline__ void join(const R (&S)[(N + 1) / 2], const R (&Dd)[N / 2],
                                     R (&out)[N]) {
  using O = EoOps<R>;
#pragma unroll
  for (int o = 0; o < N / 2; ++o) {
    out[o] = O::fin(O::add(S[o], Dd[o]));
    out[N - 1 - o] = O::fin(O::sub(S[o], Dd[o]));
  }
  if constexpr (N % 2 == 1) out[N / 2] = O::fin(S[N / 2]);
}

template <int N, class R>
__device__ __forceinline__ R dot(const R (&c)[N], const R (&u)[N]) {
  using O = EoOps<R>;
  R r = O::mul(c[0], u[0]);
#pragma unroll
  for (int i = 1; i < N; ++i) r = O::mac(c[i], u[i], r);
  return r;
}

template <int N, class R>
__device__ __forceinline__ R dot_acc(const R (&c)[N], const R (&u)[N], R r) {
  using O = EoOps<R>;
#pragma unroll
  for (int i = 0; i < N; ++i) r = O::mac(c[i], u[i], r);
  return r;
}

// r[k] (+)= c[k][q] s for the NA accumulators; the first pair initialises them
template <int NA, int NC, class R>
__device__ __forceinline__ void acc_col(R (&r)[NA], const R (&c)[NA][NC], int q, R s, bool first) {
  using O = EoOps<R>;
#pragma unroll
  for (int k = 0; k < NA; ++k) r[k] = first ? O::mul(c[k][q], s) : O::mac(c[k][q], s, r[k]);
}

// D times g at one point, D symmetric with entries (xx, xy, xz, yy, yz, zz)
template <class R>
__device__ __forceinline__ void dmul(const R (&c)[6], R g0, R g1, R g2, R& v0, R& v1, R& v2) {
  using O = EoOps<R>;
  v0 = O::fin(O::mac(c[2], g2, O::mac(c[1], g1, O::mul(c[0], g0))));
  v1 = O::fin(O::mac(c[4], g2, O::mac(c[3], g1, O::mul(c[1], g0))));
  v2 = O::fin(O::mac(c[5], g2, O::mac(c[4], g1, O::mul(c[2], g0))));
}

// ---- line contractions from the halves (outputs normalised)
// forward B: out[q] = sum_d B[q][d] v[d]
template <class R, int D, int Q>
__device__ __forceinline__ void fwd_b(const TabEO<R, D, Q>& t, const R (&ue)[(D + 1) / 2],
                                      const R (&uo)[D / 2], R (&out)[Q]) {
  R S[(Q + 1) / 2], Dd[Q / 2];
#pragma unroll
  for (int o = 0; o < (Q + 1) / 2; ++o) S[o] = dot(t.bS[o], ue);
#pragma unroll
  for (int o = 0; o < Q / 2; ++o) Dd[o] = dot(t.bD[o], uo);
  join<Q>(S, Dd, out);
}

// forward G: out[q] = sum_d G[q][d] v[d]
template <class R, int D, int Q>
__device__ __forceinline__ void fwd_g(const TabEO<R, D, Q>& t, const R (&ue)[(D + 1) / 2],
                                      const R (&uo)[D / 2], R (&out)[Q]) {
  R S[(Q + 1) / 2], Dd[Q / 2];
#pragma unroll
  for (int o = 0; o < (Q + 1) / 2; ++o) S[o] = dot(t.gS[o], uo);
#pragma unroll
  for (int o = 0; o < Q / 2; ++o) Dd[o] = dot(t.gD[o], ue);
  join<Q>(S, Dd, out);
}

// transposed B: out[d] = sum_q B[q][d] a[q], from a's halves over q
template <class R, int D, int Q>
__device__ __forceinline__ void tr_b(const TabEO<R, D, Q>& t, const R (&ae)[(Q + 1) / 2],
                                     const R (&ao)[Q / 2], R (&out)[D]) {
  R S[(D + 1) / 2], Dd[D / 2];
#pragma unroll
  for (int k = 0; k < (D + 1) / 2; ++k) S[k] = dot(t.btS[k], ae);
#pragma unroll
  for (int k = 0; k < D / 2; ++k) Dd[k] = dot(t.btD[k], ao);
  join<D>(S, Dd, out);
}

// transposed G of a plus transposed B of b: out[d] = sum_q G[q][d] a[q] + B[q][d] b[q]
template <class R, int D, int Q>
__device__ __forceinline__ void tr_gb(const TabEO<R, D, Q>& t, const R (&ae)[(Q + 1) / 2],
                                      const R (&ao)[Q / 2], const R (&be)[(Q + 1) / 2],
                                      const R (&bo)[Q / 2], R (&out)[D]) {
  R S[(D + 1) / 2], Dd[D / 2];
#pragma unroll
  for (int k = 0; k < (D + 1) / 2; ++k) S[k] = dot_acc(t.btS[k], be, dot(t.gtS[k], ao));
#pragma unroll
  for (int k = 0; k < D / 2; ++k) Dd[k] = dot_acc(t.btD[k], bo, dot(t.gtD[k], ae));
  join<D>(S, Dd, out);
}

// ---- x phase: contract i -> qx.  line (j, k); out T1c[j][k*Q + qx], c = (B x, G x).
//      Scaled policies hold the gathered FP64 values in bufA and convert them here with the
//      block's scale 2^(1023 - xexp).
template <int D, int Q, int NT, bool DIFF, class L, class Ar>
__device__ __forceinline__ void x_phase(const typename Ar::template Tab<D, Q>& tab,
                                        const typename Ar::T* bufA, typename Ar::T* bufB,
                                        int nel, int tid, int xexp) {
  using R = typename Ar::T;
  constexpr int D2 = D * D;
  for (int t = tid; t < nel * D2; t += NT) {
    const int el = t / D2, l = t - el * D2;
    const int j = l / D, k = l - j * D;
    const R* in = bufA + el * L::SZ_A + l;
    R v[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      if constexpr (Ar::kScaled)
        v[i] = Ar::from_raw(reinterpret_cast<const double*>(in)[i * L::S_DD], 1023 - xexp);
      else
        v[i] = in[i * L::S_DD];
    }
    R ue[(D + 1) / 2], uo[D / 2];
    split<D>(v, ue, uo);
    R* outb = bufB + el * L::SZ_B + j * L::S_QD + k * Q;
    R o[Q];
    fwd_b(tab, ue, uo, o);
#pragma unroll
    for (int qx = 0; qx < Q; ++qx) outb[qx] = o[qx];
    if constexpr (DIFF) {
      fwd_g(tab, ue, uo, o);
#pragma unroll
      for (int qx = 0; qx < Q; ++qx) outb[D * L::S_QD + qx] = o[qx];
    }
  }
}

// ---- y phase: contract j -> qy.  line (k, qx); out T2c[k][qy*Q + qx]
//      diffusion: c0 = B_y (G_x x), c1 = G_y (B_x x), c2 = B_y (B_x x)
template <int D, int Q, int NT, bool DIFF, class L, class Ar>
__device__ __forceinline__ void y_phase(const typename Ar::template Tab<D, Q>& tab,
                                        const typename Ar::T* bufB, typename Ar::T* bufA,
                                        int nel, int tid) {
  using R = typename Ar::T;
  constexpr int QD = Q * D;
  for (int t = tid; t < nel * QD; t += NT) {
    const int el = t / QD, l = t - el * QD;
    const int k = l / Q, qx = l - k * Q;
    const R* in = bufB + el * L::SZ_B + l;
    R vb[D];
#pragma unroll
    for (int j = 0; j < D; ++j) vb[j] = in[j * L::S_QD];
    R be[(D + 1) / 2], bo[D / 2];
    split<D>(vb, be, bo);
    R* out = bufA + el * L::SZ_A + k * L::S_QQ + qx;
    R o[Q];
    if constexpr (DIFF) {
      R vg[D];
#pragma unroll
      for (int j = 0; j < D; ++j) vg[j] = in[D * L::S_QD + j * L::S_QD];
      R ge[(D + 1) / 2], go[D / 2];
      split<D>(vg, ge, go);
      fwd_b(tab, ge, go, o);
#pragma unroll
      for (int qy = 0; qy < Q; ++qy) out[qy * Q] = o[qy];
      fwd_g(tab, be, bo, o);
#pragma unroll
      for (int qy = 0; qy < Q; ++qy) out[D * L::S_QQ + qy * Q] = o[qy];
      fwd_b(tab, be, bo, o);
#pragma unroll
      for (int qy = 0; qy < Q; ++qy) out[2 * D * L::S_QQ + qy * Q] = o[qy];
    } else {
      fwd_b(tab, be, bo, o);
#pragma unroll
      for (int qy = 0; qy < Q; ++qy) out[qy * Q] = o[qy];
    }
  }
}

// ---- z phase: contract k -> qz, apply D, contract qz -> k.  line (qy, qx); out S4c[qy][k*Q + qx]
//      The quadrature points qz and Q-1-qz are taken together: the forward contraction gives both
//      from one pair of half-size sums, and the sum and difference of their pointwise products
//      are the even and odd parts the transposed contraction needs.
template <int D, int Q, int NT, bool DIFF, class L, class Ar>
__device__ __forceinline__ void z_phase(const typename Ar::template Tab<D, Q>& tab,
                                        const typename Ar::T* bufA, typename Ar::T* bufB,
                                        const typename Ar::QdT* __restrict__ qd, int64_t e0,
                                        int nel, int tid) {
  using R = typename Ar::T;
  using O = EoOps<R>;
  constexpr int Q2 = Q * Q, DE = (D + 1) / 2, DH = D / 2, QH = Q / 2;
  constexpr int NQD = DIFF ? 6 : 1;
  for (int t = tid; t < nel * Q2; t += NT) {
    const int el = t / Q2, l = t - el * Q2;
    const int qy = l / Q, qx = l - qy * Q;
    const R* in = bufA + el * L::SZ_A + l;
    const typename Ar::QdT* qe = qd + (e0 + el) * (int64_t)(NQD * Q * Q2) + l;
    R* out = bufB + el * L::SZ_B + qy * L::S_QD + qx;
    if constexpr (DIFF) {
      R c[D];
      R e0_[DE], o0[DH], e1[DE], o1[DH], e2[DE], o2[DH];
#pragma unroll
      for (int k = 0; k < D; ++k) c[k] = in[k * L::S_QQ];
      split<D>(c, e0_, o0);
#pragma unroll
      for (int k = 0; k < D; ++k) c[k] = in[D * L::S_QQ + k * L::S_QQ];
      split<D>(c, e1, o1);
#pragma unroll
      for (int k = 0; k < D; ++k) c[k] = in[2 * D * L::S_QQ + k * L::S_QQ];
      split<D>(c, e2, o2);
      // transposed accumulators: B^T of v0 and v1, G^T of v2
      R S0[DE], D0[DH], S1[DE], D1[DH], S2[DE], D2[DH];
#pragma unroll
      for (int q = 0; q < QH; ++q) {
        const int qh = Q - 1 - q;
        R dl[6], dh[6];
#pragma unroll
        for (int cc = 0; cc < 6; ++cc) {
          dl[cc] = Ar::load_qd(qe + (q * 6 + cc) * Q2);
          dh[cc] = Ar::load_qd(qe + (qh * 6 + cc) * Q2);
        }
        const R s0 = dot(tab.bS[q], e0_), d0 = dot(tab.bD[q], o0);
        const R s1 = dot(tab.bS[q], e1), d1 = dot(tab.bD[q], o1);
        const R s2 = dot(tab.gS[q], o2), d2 = dot(tab.gD[q], e2);
        R v0l, v1l, v2l, v0h, v1h, v2h;
        dmul(dl, O::fin(O::add(s0, d0)), O::fin(O::add(s1, d1)), O::fin(O::add(s2, d2)), v0l,
             v1l, v2l);
        dmul(dh, O::fin(O::sub(s0, d0)), O::fin(O::sub(s1, d1)), O::fin(O::sub(s2, d2)), v0h,
             v1h, v2h);
        const bool first = (q == 0);
        acc_col(S0, tab.btS, q, O::add(v0l, v0h), first);
        acc_col(D0, tab.btD, q, O::sub(v0l, v0h), first);
        acc_col(S1, tab.btS, q, O::add(v1l, v1h), first);
        acc_col(D1, tab.btD, q, O::sub(v1l, v1h), first);
        acc_col(S2, tab.gtS, q, O::sub(v2l, v2h), first);
        acc_col(D2, tab.gtD, q, O::add(v2l, v2h), first);
      }
      if constexpr (Q % 2 == 1) {  // the middle point: even part only (no odd partner)
        R dm[6];
#pragma unroll
        for (int cc = 0; cc < 6; ++cc) dm[cc] = Ar::load_qd(qe + (QH * 6 + cc) * Q2);
        R v0, v1, v2;
        dmul(dm, O::fin(dot(tab.bS[QH], e0_)), O::fin(dot(tab.bS[QH], e1)),
             O::fin(dot(tab.gS[QH], o2)), v0, v1, v2);
        acc_col(S0, tab.btS, QH, v0, false);
        acc_col(S1, tab.btS, QH, v1, false);
        acc_col(D2, tab.gtD, QH, v2, false);
      }
      R w[D];
      join<D>(S0, D0, w);
#pragma unroll
      for (int k = 0; k < D; ++k) out[k * Q] = w[k];
      join<D>(S1, D1, w);
#pragma unroll
      for (int k = 0; k < D; ++k) out[Q * L::S_QD + k * Q] = w[k];
      join<D>(S2, D2, w);
#pragma unroll
      for (int k = 0; k < D; ++k) out[2 * Q * L::S_QD + k * Q] = w[k];
    } else {
      R c[D], ce[DE], co[DH];
#pragma unroll
      for (int k = 0; k < D; ++k) c[k] = in[k * L::S_QQ];
      split<D>(c, ce, co);
      R S[DE], Dd[DH];
#pragma unroll
      for (int q = 0; q < QH; ++q) {
        const R dl = Ar::load_qd(qe + q * Q2), dh = Ar::load_qd(qe + (Q - 1 - q) * Q2);
        const R s = dot(tab.bS[q], ce), d = dot(tab.bD[q], co);
        const R vl = O::fin(O::mul(dl, O::fin(O::add(s, d))));
        const R vh = O::fin(O::mul(dh, O::fin(O::sub(s, d))));
        acc_col(S, tab.btS, q, O::add(vl, vh), q == 0);
        acc_col(Dd, tab.btD, q, O::sub(vl, vh), q == 0);
      }
      if constexpr (Q % 2 == 1) {
        const R v = O::fin(O::mul(Ar::load_qd(qe + QH * Q2), O::fin(dot(tab.bS[QH], ce))));
        acc_col(S, tab.btS, QH, v, false);
      }
      R w[D];
      join<D>(S, Dd, w);
#pragma unroll
      for (int k = 0; k < D; ++k) out[k * Q] = w[k];
    }
  }
}

// ---- y^T phase: contract qy -> j.  line (k, qx); out S5c[qx][j*D + k]
//      diffusion: c0 (-> G_x^T) = B_y^T s0, c1 (-> B_x^T) = G_y^T s1 + B_y^T s2
template <int D, int Q, int NT, bool DIFF, class L, class Ar>
__device__ __forceinline__ void yt_phase(const typename Ar::template Tab<D, Q>& tab,
                                         const typename Ar::T* bufB, typename Ar::T* bufA,
                                         int nel, int tid) {
  using R = typename Ar::T;
  constexpr int QD = Q * D, QE = (Q + 1) / 2, QH = Q / 2;
  for (int t = tid; t < nel * QD; t += NT) {
    const int el = t / QD, l = t - el * QD;
    const int k = l / Q, qx = l - k * Q;
    const R* in = bufB + el * L::SZ_B + l;
    R* out = bufA + el * L::SZ_A + qx * L::S_DD + k;
    R a[Q], ae[QE], ao[QH], r[D];
#pragma unroll
    for (int qy = 0; qy < Q; ++qy) a[qy] = in[qy * L::S_QD];
    split<Q>(a, ae, ao);
    tr_b(tab, ae, ao, r);
#pragma unroll
    for (int j = 0; j < D; ++j) out[j * D] = r[j];
    if constexpr (DIFF) {
      R be[QE], bo[QH];
#pragma unroll
      for (int qy = 0; qy < Q; ++qy) a[qy] = in[Q * L::S_QD + qy * L::S_QD];
      split<Q>(a, ae, ao);
#pragma unroll
      for (int qy = 0; qy < Q; ++qy) a[qy] = in[2 * Q * L::S_QD + qy * L::S_QD];
      split<Q>(a, be, bo);
      tr_gb(tab, ae, ao, be, bo, r);
#pragma unroll
      for (int j = 0; j < D; ++j) out[Q * L::S_DD + j * D] = r[j];
    }
  }
}

// ---- x^T phase: contract qx -> i.  line (j, k); out Ye[i + D j + D^2 k]
//      diffusion: G_x^T of the first array plus B_x^T of the second; mass: B_x^T
template <int D, int Q, int NT, bool DIFF, class L, class Ar>
__device__ __forceinline__ void xt_phase(const typename Ar::template Tab<D, Q>& tab,
                                         const typename Ar::T* bufA, typename Ar::T* bufB,
                                         int nel, int tid) {
  using R = typename Ar::T;
  constexpr int D2 = D * D, QE = (Q + 1) / 2, QH = Q / 2;
  for (int t = tid; t < nel * D2; t += NT) {
    const int el = t / D2, l = t - el * D2;
    const int j = l / D, k = l - j * D;
    const R* in = bufA + el * L::SZ_A + l;
    R a[Q], ae[QE], ao[QH], r[D];
#pragma unroll
    for (int qx = 0; qx < Q; ++qx) a[qx] = in[qx * L::S_DD];
    split<Q>(a, ae, ao);
    if constexpr (DIFF) {
      R be[QE], bo[QH];
#pragma unroll
      for (int qx = 0; qx < Q; ++qx) a[qx] = in[Q * L::S_DD + qx * L::S_DD];
      split<Q>(a, be, bo);
      tr_gb(tab, ae, ao, be, bo, r);
    } else {
      tr_b(tab, ae, ao, r);
    }
    R* out = bufB + el * L::SZ_B + j * D + k * D2;
#pragma unroll
    for (int i = 0; i < D; ++i) out[i] = r[i];
  }
}

}  // namespace eo
}  // namespace fe
