// The paper's own operator: the mixed H1 / L2 gradient and divergence blocks of the
// acoustic-gravity system (Section II-A, Eq. (block-mult): (grad p, tau) and -(u, grad v)),
// applied in partial-assembly form by one fused kernel (Section III-G: both blocks share the
// geometric factors at the quadrature points, so one pass over the elements reads them once).
//
// Spaces (readings; the paper fixes only the orders): pressure in continuous H1 of order p_h on
// Gauss-Lobatto-Legendre nodes with the structured mesh's dof map; velocity in discontinuous L2
// of order p_l, one Lagrange basis per element on the p_l + 1 Gauss-Legendre points per axis,
// three components, layout [e][c][a], a = i + D_l (j + D_l k); Q = p_h + 1 Gauss-Legendre points
// per axis; the L2 basis is used as is on the physical element.  Then
//   (G p)_{e,c,a} = sum_q psi_a(x_q) sum_r M_q[c][r] (d p / d xi_r)(x_q),
//   M_q = w_q det J J^-T = w_q adj(J)^T,
// and the divergence block is G^T.  Per element the kernel takes the pressure through the
// reference gradient (the sum-factorised B/G contractions of Eq. (2), as in the diffusion apply),
// applies M_q, and the L2 test basis transposed; and the velocity through the L2 basis, M_q^T,
// and the transposed reference gradient, scatter-added into the H1 vector.  FP64 FMA throughout
// (on GB300 the FP64 tensor instruction is slower per flop than FP64 FMA, so no DMMA path); every
// 1D contraction on the even and odd halves of its line (the tables' reversal symmetry, as in the
// diffusion apply: fe_apply_eo.cuh), which cuts the FP64 instructions that bound the kernel.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "fe_apply_eo.cuh"
#include "fe_internal.h"

struct fe_mixed {
  int nx = 0, ny = 0, nz = 0, ph = 0, pl = 0, Dh = 0, Dl = 0, Q = 0;
  int64_t ne = 0, ndof_h = 0, ndof_l = 0;
  fe_mesh* mesh = nullptr;  // H1 dof map and vertices (owned)
  double* d_qd = nullptr;   // [ne][qz][9][qy][qx]: M_q[c][r] at m = 3 c + r
  double Bh[fe::kMaxQ * fe::kMaxD], Gh[fe::kMaxQ * fe::kMaxD], Bl[fe::kMaxQ * fe::kMaxD];
  double pts[fe::kMaxQ], wts[fe::kMaxQ];
};

namespace {

using namespace fe;

constexpr int kNT = 128;               // threads per block
constexpr int kSmem = 96 * 1024;       // shared-memory budget per block

__host__ __device__ constexpr int oddp(int n) { return (n % 2 == 0) ? n + 1 : n; }
__host__ __device__ constexpr int cmx(int a, int b) { return a > b ? a : b; }

// H1 tables (B_h, G_h) and the L2 table (B_l, its G unused), with their even-odd halves
template <int DH, int DL, int Q>
struct MixedTab {
  TabEO<double, DH, Q> h;
  TabEO<double, DL, Q> l;
};

// Shared-memory layout per element (doubles).  Every array stores the summed index of the next
// phase slowest, with odd-padded slabs.  Buffer A: the gathered inputs, then the y-phase
// outputs, then the transposed-y outputs; buffer B: the x-phase outputs, then the z-phase ones.
template <int DH, int DL, int Q>
struct MixedLayout {
  static constexpr int hDD = oddp(DH * DH), lDD = oddp(DL * DL);
  static constexpr int hQD = oddp(Q * DH), lQD = oddp(Q * DL), QQ = oddp(Q * Q);
  static constexpr int A_U = DH * hDD, A1 = A_U + 3 * DL * lDD;        // P [i][j,k], U [c][i][j,k]
  static constexpr int A_YL = 3 * DH * QQ, A3 = A_YL + 3 * DL * QQ;    // YH [c][k][qy,qx], YL
  static constexpr int A_WL = 2 * Q * hDD, A5 = A_WL + 3 * Q * lDD;    // WH [c][qx][j,k], WL
  static constexpr int SA = cmx(A1, cmx(A3, A5));
  static constexpr int B_TL = 2 * DH * hQD, B2 = B_TL + 3 * DL * lQD;  // TH [c][j][k,qx], TL
  static constexpr int B_ZL = 3 * Q * hQD, B4 = B_ZL + 3 * Q * lQD;    // ZH [c][qy][k,qx], ZL
  static constexpr int SB = cmx(B2, B4);
  static constexpr int PER = SA + SB;
  static constexpr int NE = kSmem / (PER * 8) < 1 ? 1 : kSmem / (PER * 8);
};

// GRAD: gp = G p; DIV: gtu = G^T u (gtu zeroed by the caller: atomic scatter-add).
template <int DH, int DL, int Q, bool GRAD, bool DIV>
__global__ void __launch_bounds__(kNT) k_mixed_apply(const int32_t* __restrict__ map,
                                                     const double* __restrict__ qd,
                                                     const double* __restrict__ p,
                                                     const double* __restrict__ u,
                                                     double* __restrict__ gp,
                                                     double* __restrict__ gtu, int64_t ne,
                                                     const MixedTab<DH, DL, Q> tab) {
  using L = MixedLayout<DH, DL, Q>;
  constexpr int NE = L::NE;
  constexpr int DH2 = DH * DH, DH3 = DH2 * DH, DL2 = DL * DL, DL3 = DL2 * DL, Q2 = Q * Q;
  constexpr int hDD = L::hDD, lDD = L::lDD, hQD = L::hQD, lQD = L::lQD, QQ = L::QQ;
  constexpr int DHE = (DH + 1) / 2, DHH = DH / 2, DLE = (DL + 1) / 2, DLH = DL / 2;
  constexpr int QE = (Q + 1) / 2, QH = Q / 2;
  extern __shared__ __align__(16) double sm[];
  double* bufA = sm;
  double* bufB = sm + NE * L::SA;
  const int64_t e0 = (int64_t)blockIdx.x * NE;
  const int nel = (int)((ne - e0) < NE ? (ne - e0) : NE);
  const int tid = threadIdx.x;

  // ---- gather: P[i][j*DH + k] = p[map[e][i + DH j + DH^2 k]]; U[c][i][j*DL + k] = u[e][c][a]
  if constexpr (GRAD) {
    for (int t = tid; t < nel * DH3; t += kNT) {
      const int el = t / DH3, a = t - el * DH3;
      const int i = a % DH, j = (a / DH) % DH, k = a / DH2;
      bufA[el * L::SA + i * hDD + j * DH + k] = __ldg(&p[__ldg(&map[(e0 + el) * DH3 + a])]);
    }
  }
  if constexpr (DIV) {
    for (int t = tid; t < nel * 3 * DL3; t += kNT) {
      const int el = t / (3 * DL3), r = t - el * 3 * DL3, c = r / DL3, a = r - c * DL3;
      const int i = a % DL, j = (a / DL) % DL, k = a / DL2;
      bufA[el * L::SA + L::A_U + (c * DL + i) * lDD + j * DL + k] = __ldg(&u[(e0 + el) * 3 * DL3 + r]);
    }
  }
  __syncthreads();

  // ---- x phase.  H1 lines (j, k): TH[0] = B_h x, TH[1] = G_h x along i; L2 lines (c, j, k)
  if constexpr (GRAD) {
    for (int t = tid; t < nel * DH2; t += kNT) {
      const int el = t / DH2, l = t - el * DH2, j = l / DH, k = l - j * DH;
      const double* in = bufA + el * L::SA + l;
      double v[DH], ve[DHE], vo[DHH], o[Q];
#pragma unroll
      for (int i = 0; i < DH; ++i) v[i] = in[i * hDD];
      eo::split<DH>(v, ve, vo);
      double* out = bufB + el * L::SB + j * hQD + k * Q;
      eo::fwd_b(tab.h, ve, vo, o);
#pragma unroll
      for (int qx = 0; qx < Q; ++qx) out[qx] = o[qx];
      eo::fwd_g(tab.h, ve, vo, o);
#pragma unroll
      for (int qx = 0; qx < Q; ++qx) out[DH * hQD + qx] = o[qx];
    }
  }
  if constexpr (DIV) {
    for (int t = tid; t < nel * 3 * DL2; t += kNT) {
      const int el = t / (3 * DL2), r = t - el * 3 * DL2, c = r / DL2, l = r - c * DL2;
      const int j = l / DL, k = l - j * DL;
      const double* in = bufA + el * L::SA + L::A_U + c * DL * lDD + l;
      double v[DL], ve[DLE], vo[DLH], o[Q];
#pragma unroll
      for (int i = 0; i < DL; ++i) v[i] = in[i * lDD];
      eo::split<DL>(v, ve, vo);
      eo::fwd_b(tab.l, ve, vo, o);
      double* out = bufB + el * L::SB + L::B_TL + (c * DL + j) * lQD + k * Q;
#pragma unroll
      for (int qx = 0; qx < Q; ++qx) out[qx] = o[qx];
    }
  }
  __syncthreads();

  // ---- y phase.  H1 lines (k, qx): YH[0] = B_y G_x p, YH[1] = G_y B_x p, YH[2] = B_y B_x p;
  //      L2 lines (c, k, qx): YL[c] = B_l,y B_l,x u_c
  if constexpr (GRAD) {
    for (int t = tid; t < nel * DH * Q; t += kNT) {
      const int el = t / (DH * Q), l = t - el * DH * Q, k = l / Q, qx = l - k * Q;
      const double* in = bufB + el * L::SB + l;
      double vb[DH], vg[DH], be[DHE], bo[DHH], ge[DHE], go[DHH], o[Q];
#pragma unroll
      for (int j = 0; j < DH; ++j) {
        vb[j] = in[j * hQD];
        vg[j] = in[(DH + j) * hQD];
      }
      eo::split<DH>(vb, be, bo);
      eo::split<DH>(vg, ge, go);
      double* out = bufA + el * L::SA + k * QQ + qx;
      eo::fwd_b(tab.h, ge, go, o);
#pragma unroll
      for (int qy = 0; qy < Q; ++qy) out[qy * Q] = o[qy];
      eo::fwd_g(tab.h, be, bo, o);
#pragma unroll
      for (int qy = 0; qy < Q; ++qy) out[DH * QQ + qy * Q] = o[qy];
      eo::fwd_b(tab.h, be, bo, o);
#pragma unroll
      for (int qy = 0; qy < Q; ++qy) out[2 * DH * QQ + qy * Q] = o[qy];
    }
  }
  if constexpr (DIV) {
    for (int t = tid; t < nel * 3 * DL * Q; t += kNT) {
      const int el = t / (3 * DL * Q), r = t - el * 3 * DL * Q, c = r / (DL * Q);
      const int l = r - c * DL * Q, k = l / Q, qx = l - k * Q;
      const double* in = bufB + el * L::SB + L::B_TL + c * DL * lQD + l;
      double v[DL], ve[DLE], vo[DLH], o[Q];
#pragma unroll
      for (int j = 0; j < DL; ++j) v[j] = in[j * lQD];
      eo::split<DL>(v, ve, vo);
      eo::fwd_b(tab.l, ve, vo, o);
      double* out = bufA + el * L::SA + L::A_YL + (c * DL + k) * QQ + qx;
#pragma unroll
      for (int qy = 0; qy < Q; ++qy) out[qy * Q] = o[qy];
    }
  }
  __syncthreads();

  // ---- z phase, one (qy, qx) column per thread: the z contractions forward, M_q (gradient) and
  //      M_q^T (divergence) at every qz, and the transposed z contractions, in registers.  The
  //      points qz and Q-1-qz are taken together (even-odd halves, as in the diffusion apply).
  for (int t = tid; t < nel * Q2; t += kNT) {
    const int el = t / Q2, l = t - el * Q2, qy = l / Q, qx = l - qy * Q;
    const int ls = qy * Q + qx;  // (qy, qx) in the padded slabs (same as l: QQ slabs)
    const double* qe = qd + (e0 + el) * (int64_t)(9 * Q * Q2) + l;
    // gradient: H1 inputs' halves, L2 transposed accumulators (S on even, D on odd parts)
    double he[3][DHE], ho[3][DHH], SL[3][DLE], DLa[3][DLH];
    // divergence: L2 inputs' halves, H1 transposed accumulators (G^T for component 2)
    double le[3][DLE], lo[3][DLH], SH[3][DHE], DHa[3][DHH];
    if constexpr (GRAD) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        double v[DH];
#pragma unroll
        for (int k = 0; k < DH; ++k) v[k] = bufA[el * L::SA + (c * DH + k) * QQ + ls];
        eo::split<DH>(v, he[c], ho[c]);
      }
    }
    if constexpr (DIV) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        double v[DL];
#pragma unroll
        for (int k = 0; k < DL; ++k) v[k] = bufA[el * L::SA + L::A_YL + (c * DL + k) * QQ + ls];
        eo::split<DL>(v, le[c], lo[c]);
      }
    }
#pragma unroll
    for (int q = 0; q < QH; ++q) {
      const int qh = Q - 1 - q;
      double Ml[9], Mh[9];
#pragma unroll
      for (int m = 0; m < 9; ++m) {
        Ml[m] = __ldcs(&qe[(q * 9 + m) * Q2]);
        Mh[m] = __ldcs(&qe[(qh * 9 + m) * Q2]);
      }
      const bool first = (q == 0);
      if constexpr (GRAD) {
        const double s0 = eo::dot(tab.h.bS[q], he[0]), d0 = eo::dot(tab.h.bD[q], ho[0]);
        const double s1 = eo::dot(tab.h.bS[q], he[1]), d1 = eo::dot(tab.h.bD[q], ho[1]);
        const double s2 = eo::dot(tab.h.gS[q], ho[2]), d2 = eo::dot(tab.h.gD[q], he[2]);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const double vl = fma(Ml[3 * c + 2], s2 + d2, fma(Ml[3 * c + 1], s1 + d1, Ml[3 * c] * (s0 + d0)));
          const double vh = fma(Mh[3 * c + 2], s2 - d2, fma(Mh[3 * c + 1], s1 - d1, Mh[3 * c] * (s0 - d0)));
          eo::acc_col(SL[c], tab.l.btS, q, vl + vh, first);
          eo::acc_col(DLa[c], tab.l.btD, q, vl - vh, first);
        }
      }
      if constexpr (DIV) {
        double ul[3], uh[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const double s = eo::dot(tab.l.bS[q], le[c]), d = eo::dot(tab.l.bD[q], lo[c]);
          ul[c] = s + d;
          uh[c] = s - d;
        }
        double wl[3], wh[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          wl[r] = fma(Ml[6 + r], ul[2], fma(Ml[3 + r], ul[1], Ml[r] * ul[0]));
          wh[r] = fma(Mh[6 + r], uh[2], fma(Mh[3 + r], uh[1], Mh[r] * uh[0]));
        }
        eo::acc_col(SH[0], tab.h.btS, q, wl[0] + wh[0], first);
        eo::acc_col(DHa[0], tab.h.btD, q, wl[0] - wh[0], first);
        eo::acc_col(SH[1], tab.h.btS, q, wl[1] + wh[1], first);
        eo::acc_col(DHa[1], tab.h.btD, q, wl[1] - wh[1], first);
        eo::acc_col(SH[2], tab.h.gtS, q, wl[2] - wh[2], first);
        eo::acc_col(DHa[2], tab.h.gtD, q, wl[2] + wh[2], first);
      }
    }
    if constexpr (Q % 2 == 1) {  // the middle point: even parts only
      double M[9];
#pragma unroll
      for (int m = 0; m < 9; ++m) M[m] = __ldcs(&qe[(QH * 9 + m) * Q2]);
      if constexpr (GRAD) {
        const double g0 = eo::dot(tab.h.bS[QH], he[0]), g1 = eo::dot(tab.h.bS[QH], he[1]);
        const double g2 = eo::dot(tab.h.gS[QH], ho[2]);
#pragma unroll
        for (int c = 0; c < 3; ++c)
          eo::acc_col(SL[c], tab.l.btS, QH, fma(M[3 * c + 2], g2, fma(M[3 * c + 1], g1, M[3 * c] * g0)), false);
      }
      if constexpr (DIV) {
        double u[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) u[c] = eo::dot(tab.l.bS[QH], le[c]);
        eo::acc_col(SH[0], tab.h.btS, QH, fma(M[6], u[2], fma(M[3], u[1], M[0] * u[0])), false);
        eo::acc_col(SH[1], tab.h.btS, QH, fma(M[7], u[2], fma(M[4], u[1], M[1] * u[0])), false);
        eo::acc_col(DHa[2], tab.h.gtD, QH, fma(M[8], u[2], fma(M[5], u[1], M[2] * u[0])), false);
      }
    }
    if constexpr (GRAD) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        double w[DL];
        eo::join<DL>(SL[c], DLa[c], w);
#pragma unroll
        for (int k = 0; k < DL; ++k)
          bufB[el * L::SB + L::B_ZL + (c * Q + qy) * lQD + k * Q + qx] = w[k];
      }
    }
    if constexpr (DIV) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        double w[DH];
        eo::join<DH>(SH[c], DHa[c], w);
#pragma unroll
        for (int k = 0; k < DH; ++k) bufB[el * L::SB + (c * Q + qy) * hQD + k * Q + qx] = w[k];
      }
    }
  }
  __syncthreads();

  // ---- transposed y.  H1 lines (k, qx): WH[0] = B_y^T ZH[0], WH[1] = G_y^T ZH[1] + B_y^T ZH[2];
  //      L2 lines (c, k, qx): WL[c] = B_l,y^T ZL[c]
  if constexpr (DIV) {
    for (int t = tid; t < nel * DH * Q; t += kNT) {
      const int el = t / (DH * Q), l = t - el * DH * Q, k = l / Q, qx = l - k * Q;
      const double* in = bufB + el * L::SB + l;
      double a[Q], ae[QE], ao[QH], be[QE], bo[QH], r[DH];
#pragma unroll
      for (int qy = 0; qy < Q; ++qy) a[qy] = in[qy * hQD];
      eo::split<Q>(a, ae, ao);
      double* out = bufA + el * L::SA + qx * hDD + k;
      eo::tr_b(tab.h, ae, ao, r);
#pragma unroll
      for (int j = 0; j < DH; ++j) out[j * DH] = r[j];
#pragma unroll
      for (int qy = 0; qy < Q; ++qy) a[qy] = in[(Q + qy) * hQD];
      eo::split<Q>(a, ae, ao);
#pragma unroll
      for (int qy = 0; qy < Q; ++qy) a[qy] = in[(2 * Q + qy) * hQD];
      eo::split<Q>(a, be, bo);
      eo::tr_gb(tab.h, ae, ao, be, bo, r);
#pragma unroll
      for (int j = 0; j < DH; ++j) out[Q * hDD + j * DH] = r[j];
    }
  }
  if constexpr (GRAD) {
    for (int t = tid; t < nel * 3 * DL * Q; t += kNT) {
      const int el = t / (3 * DL * Q), r = t - el * 3 * DL * Q, c = r / (DL * Q);
      const int l = r - c * DL * Q, k = l / Q, qx = l - k * Q;
      const double* in = bufB + el * L::SB + L::B_ZL + c * Q * lQD + l;
      double a[Q], ae[QE], ao[QH], acc[DL];
#pragma unroll
      for (int qy = 0; qy < Q; ++qy) a[qy] = in[qy * lQD];
      eo::split<Q>(a, ae, ao);
      eo::tr_b(tab.l, ae, ao, acc);
      double* out = bufA + el * L::SA + L::A_WL + (c * Q + qx) * lDD + k;
#pragma unroll
      for (int j = 0; j < DL; ++j) out[j * DL] = acc[j];
    }
  }
  __syncthreads();

  // ---- transposed x and the outputs.  H1 lines (j, k): G_x^T WH[0] + B_x^T WH[1], scatter-added
  //      into gtu; L2 lines (c, j, k), j fastest: B_l,x^T WL[c], written to gp[e][c][i + DL l]
  if constexpr (DIV) {
    for (int t = tid; t < nel * DH2; t += kNT) {
      const int el = t / DH2, l = t - el * DH2, j = l / DH, k = l - j * DH;
      const double* in = bufA + el * L::SA + j * DH + k;
      double a[Q], ae[QE], ao[QH], be[QE], bo[QH], r[DH];
#pragma unroll
      for (int qx = 0; qx < Q; ++qx) a[qx] = in[qx * hDD];
      eo::split<Q>(a, ae, ao);
#pragma unroll
      for (int qx = 0; qx < Q; ++qx) a[qx] = in[(Q + qx) * hDD];
      eo::split<Q>(a, be, bo);
      eo::tr_gb(tab.h, ae, ao, be, bo, r);
      const int32_t* me = map + (e0 + el) * DH3 + j * DH + k * DH2;
#pragma unroll
      for (int i = 0; i < DH; ++i) atomicAdd(&gtu[__ldg(&me[i])], r[i]);
    }
  }
  if constexpr (GRAD) {
    for (int t = tid; t < nel * 3 * DL2; t += kNT) {
      const int el = t / (3 * DL2), r = t - el * 3 * DL2, c = r / DL2, l = r - c * DL2;
      const int k = l / DL, j = l - k * DL;  // j fastest: consecutive threads, consecutive rows
      const double* in = bufA + el * L::SA + L::A_WL + c * Q * lDD + j * DL + k;
      double a[Q], ae[QE], ao[QH], acc[DL];
#pragma unroll
      for (int qx = 0; qx < Q; ++qx) a[qx] = in[qx * lDD];
      eo::split<Q>(a, ae, ao);
      eo::tr_b(tab.l, ae, ao, acc);
      double* out = gp + ((e0 + el) * 3 + c) * DL3 + (j + DL * k) * DL;
#pragma unroll
      for (int i = 0; i < DL; ++i) out[i] = acc[i];
    }
  }
}

// PA data of the pair: M_q = w_q adj(J)^T at every element and Gauss point, stored
// [e][qz][9][qy][qx] with m = 3 c + r; counts points with det J <= 0 in *bad.
struct Rule1D {
  double pts[kMaxQ], wts[kMaxQ];
};

__global__ void k_mixed_qdata(const double* __restrict__ V, int nx, int ny, int64_t ne, int Q,
                              const Rule1D rule, double* __restrict__ qd, int* bad) {
  const int Q2 = Q * Q, Q3 = Q2 * Q;
  const int64_t n = ne * Q3;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = t / Q3;
    const int q = (int)(t - e * Q3), qx = q % Q, qy = (q / Q) % Q, qz = q / Q2;
    const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((int64_t)nx * ny));
    const double s = rule.pts[qx], tt = rule.pts[qy], uu = rule.pts[qz];
    double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int v = 0; v < 8; ++v) {
      const int a = v & 1, b = (v >> 1) & 1, c = v >> 2;
      const int64_t idx = (ex + a) + (int64_t)(nx + 1) * ((ey + b) + (int64_t)(ny + 1) * (ez + c));
      const double fa = a ? s : 1.0 - s, fb = b ? tt : 1.0 - tt, fc = c ? uu : 1.0 - uu;
      const double dN[3] = {(a ? 1.0 : -1.0) * fb * fc, fa * (b ? 1.0 : -1.0) * fc,
                            fa * fb * (c ? 1.0 : -1.0)};
      for (int i = 0; i < 3; ++i) {
        const double xv = V[3 * idx + i];
        for (int r = 0; r < 3; ++r) J[i][r] = fma(xv, dN[r], J[i][r]);
      }
    }
    // adj[r][i]: cofactor of J[i][r] (adj(J) = det J J^-1)
    double adj[3][3];
    adj[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    adj[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    adj[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    adj[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    adj[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    adj[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    adj[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    adj[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    adj[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    const double det = J[0][0] * adj[0][0] + J[0][1] * adj[1][0] + J[0][2] * adj[2][0];
    if (!(det > 0.0)) atomicAdd(bad, 1);
    const double w = rule.wts[qx] * rule.wts[qy] * rule.wts[qz];
    double* out = qd + e * (int64_t)(9 * Q3) + (int64_t)qz * 9 * Q2 + qy * Q + qx;
    for (int c = 0; c < 3; ++c)
      for (int r = 0; r < 3; ++r) out[(3 * c + r) * Q2] = w * adj[r][c];  // (w det J J^-T)[c][r]
  }
}

template <int DH, int DL, int Q, bool GRAD, bool DIV>
int launch_mixed(const fe_mixed* mx, const double* p, const double* u, double* gp, double* gtu,
                 cudaStream_t s) {
  using L = MixedLayout<DH, DL, Q>;
  auto kern = k_mixed_apply<DH, DL, Q, GRAD, DIV>;
  const size_t smem = (size_t)L::NE * L::PER * sizeof(double);
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [&] {
    attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (attr != cudaSuccess) return cuda_error(attr, "fe_mixed_apply: cudaFuncSetAttribute");
  MixedTab<DH, DL, Q> tab;
  eo::fill(mx->Bh, mx->Gh, &tab.h);
  eo::fill(mx->Bl, nullptr, &tab.l);
  const int64_t nblk = (mx->ne + L::NE - 1) / L::NE;
  if (nblk == 0) return FE_OK;
  kern<<<(unsigned int)nblk, kNT, smem, s>>>(mx->mesh->d_map, mx->d_qd, p, u, gp, gtu, mx->ne,
                                               tab);
  return cuda_error(cudaGetLastError(), "fe_mixed_apply: launch");
}

template <int DH, int DL, int Q>
int dispatch_blocks(const fe_mixed* mx, const double* p, const double* u, double* gp,
                    double* gtu, cudaStream_t s) {
  const bool grad = p && gp, div = u && gtu;
  if (grad && div) return launch_mixed<DH, DL, Q, true, true>(mx, p, u, gp, gtu, s);
  if (grad) return launch_mixed<DH, DL, Q, true, false>(mx, p, u, gp, gtu, s);
  if (div) return launch_mixed<DH, DL, Q, false, true>(mx, p, u, gp, gtu, s);
  return FE_OK;
}

}  // namespace

extern "C" {

int fe_mixed_setup(int nx, int ny, int nz, int order_h, int order_l, const double* host_vertices,
                   void* stream, fe_mixed** out) {
  clear_error();
  if (!out) return set_error(FE_ERR_ARG, "fe_mixed_setup: out is NULL");
  *out = nullptr;
  const bool built = (order_h == 4 && order_l == 3) || (order_h == 2 && order_l == 1) ||
                     (order_h == 3 && order_l == 3);
  if (!built)
    return set_error(FE_ERR_UNSUPPORTED, "fe_mixed_setup: (order_h, order_l) must be (4, 3), "
                                         "(2, 1) or (3, 3)");
  fe_mixed* mx = new fe_mixed();
  int st = fe_mesh_setup(nx, ny, nz, order_h, host_vertices, &mx->mesh);
  if (st != FE_OK) {
    delete mx;
    return st;
  }
  mx->nx = nx;
  mx->ny = ny;
  mx->nz = nz;
  mx->ph = order_h;
  mx->pl = order_l;
  mx->Dh = order_h + 1;
  mx->Dl = order_l + 1;
  mx->Q = order_h + 1;
  mx->ne = mx->mesh->ne;
  mx->ndof_h = mx->mesh->ndofs;
  mx->ndof_l = mx->ne * 3 * mx->Dl * mx->Dl * mx->Dl;
  Basis1D bh;
  if (!make_basis_1d(order_h, mx->Q, &bh) || !make_l2_basis_1d(order_l, mx->Q, mx->Bl)) {
    fe_mixed_destroy(mx);
    return set_error(FE_ERR_ARG, "fe_mixed_setup: basis tables");
  }
  for (int i = 0; i < mx->Q * mx->Dh; ++i) {
    mx->Bh[i] = bh.B[i];
    mx->Gh[i] = bh.G[i];
  }
  Rule1D rule;
  for (int i = 0; i < mx->Q; ++i) {
    rule.pts[i] = mx->pts[i] = bh.pts[i];
    rule.wts[i] = mx->wts[i] = bh.wts[i];
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t nq = mx->ne * (int64_t)mx->Q * mx->Q * mx->Q;
  int* d_bad = nullptr;
  cudaError_t err;
  if ((err = cudaMalloc(&mx->d_qd, sizeof(double) * 9 * (nq > 0 ? nq : 1))) != cudaSuccess ||
      (err = cudaMalloc(&d_bad, sizeof(int))) != cudaSuccess) {
    cudaFree(d_bad);
    fe_mixed_destroy(mx);
    return cuda_error(err, "fe_mixed_setup: cudaMalloc");
  }
  int bad = 0;
  cudaMemsetAsync(d_bad, 0, sizeof(int), s);
  if (nq > 0)
    k_mixed_qdata<<<1024, 256, 0, s>>>(mx->mesh->d_vertices, nx, ny, mx->ne, mx->Q, rule,
                                       mx->d_qd, d_bad);
  if ((err = cudaGetLastError()) == cudaSuccess &&
      (err = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s)) == cudaSuccess)
    err = cudaStreamSynchronize(s);
  cudaFree(d_bad);
  if (err != cudaSuccess) {
    fe_mixed_destroy(mx);
    return cuda_error(err, "fe_mixed_setup: quadrature data");
  }
  if (bad) {
    fe_mixed_destroy(mx);
    return set_error(FE_ERR_ARG, "fe_mixed_setup: inverted element (det J <= 0 at " +
                                     std::to_string(bad) + " points)");
  }
  *out = mx;
  return FE_OK;
}

int fe_mixed_sizes(const fe_mixed* mx, int64_t* ndof_h, int64_t* ndof_l) {
  clear_error();
  if (!mx) return set_error(FE_ERR_ARG, "fe_mixed_sizes: handle is NULL");
  if (ndof_h) *ndof_h = mx->ndof_h;
  if (ndof_l) *ndof_l = mx->ndof_l;
  return FE_OK;
}

int fe_mixed_apply(const fe_mixed* mx, const double* dev_p, const double* dev_u, double* dev_gp,
                   double* dev_gtu, void* stream) {
  clear_error();
  if (!mx) return set_error(FE_ERR_ARG, "fe_mixed_apply: handle is NULL");
  if ((dev_p == nullptr) != (dev_gp == nullptr) || (dev_u == nullptr) != (dev_gtu == nullptr))
    return set_error(FE_ERR_ARG, "fe_mixed_apply: give p with gp and u with gtu (or neither)");
  cudaStream_t s = (cudaStream_t)stream;
  if (dev_gtu) {
    const cudaError_t err = cudaMemsetAsync(dev_gtu, 0, sizeof(double) * mx->ndof_h, s);
    if (err != cudaSuccess) return cuda_error(err, "fe_mixed_apply: zero gtu");
  }
  if (mx->ph == 4 && mx->pl == 3) return dispatch_blocks<5, 4, 5>(mx, dev_p, dev_u, dev_gp, dev_gtu, s);
  if (mx->ph == 2 && mx->pl == 1) return dispatch_blocks<3, 2, 3>(mx, dev_p, dev_u, dev_gp, dev_gtu, s);
  return dispatch_blocks<4, 4, 4>(mx, dev_p, dev_u, dev_gp, dev_gtu, s);
}

void fe_mixed_destroy(fe_mixed* mx) {
  if (!mx) return;
  cudaFree(mx->d_qd);
  fe_mesh_destroy(mx->mesh);
  delete mx;
}

}  // extern "C"
