// Fused partial-assembly apply kernels: y += G^T B^T D B G x for NE elements per thread block.
//
// One launch performs every step of Eq. (1) on one GPU (P = identity), fused as in
// Section III-G so that no E-vector or Q-vector ever reaches HBM:
//   gather (G):      element dofs through the dof map into shared memory;
//   B, 3 times:      sum-factorised 1D contractions (Eq. (2)), one direction per phase;
//   D:               pointwise product with the stored quadrature data (partial assembly);
//   B^T, 3 times:    the transposed contractions;
//   scatter (G^T):   atomic FP64 add into y (the "atomic write-back" of Section III-G).
//
// Work mapping (GB300-first, not the paper's one-thread-per-output-of-C layout): every phase is
// a set of independent 1D "lines" -- a line holds the D (or Q) values along the summed index
// for one position of the two other indices -- and the lines of all NE elements of the block
// are dealt out flat to the NT threads, so that warps stay full whatever D and Q are.  A thread
// keeps its line in registers, contracts it against the 1D tables (kernel parameters, read as
// constant-bank operands) and writes the results where the next phase's lines are contiguous.
// Shared-memory arrays are stored "summed index slowest" with padded slabs and per-element
// strides chosen (by a model of every phase's warp accesses, fe_smem_layout.h) to keep bank
// conflicts low -- the concern of Sections III-C/D, solved by layout rather than fragment maps.
// The z-direction phase fuses the forward z contraction, the pointwise D and the transposed z
// contraction in registers, one (qx, qy) column per thread.
#pragma once

#include <type_traits>

#include "fe_apply_eo.cuh"
#include "fe_arith.cuh"
#include "fe_smem_layout.h"

namespace fe {

__host__ __device__ constexpr int odd_pad(int n) { return (n % 2 == 0) ? n + 1 : n; }
__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }

// Field f (0 S_DD, 1 S_QD, 2 S_QQ, 3 SZ_A, 4 SZ_B) of the generated bank-conflict-minimising
// layout for (D, Q, operator, element bytes, z re-read), or 0 when the table has none.
__host__ __device__ constexpr int tuned_layout(int D, int Q, bool diff, int es, bool rr, int f) {
  for (const SmemLayoutEntry& e : kSmemLayouts) {
    if (e.D == D && e.Q == Q && e.diff == (diff ? 1 : 0) && e.es == es && e.rr == (rr ? 1 : 0)) {
      return f == 0 ? e.s_dd : f == 1 ? e.s_qd : f == 2 ? e.s_qq : f == 3 ? e.sz_a : e.sz_b;
    }
  }
  return 0;
}

// Shared-memory strides (in elements of ES bytes): the slabs are padded to an odd number of
// elements by default; ES != 0 selects the generated layout for that element size and z re-read
// mode when there is one (fe_smem_layout.h, from smem_layout.py's model of the warp accesses).
template <int D, int Q, bool DIFF, int ES = 0, bool RR = false>
struct ApplyLayout {
  static constexpr int D2 = D * D, D3 = D * D * D, Q2 = Q * Q, QD = Q * D;
  static constexpr int TUNED = ES ? tuned_layout(D, Q, DIFF, ES, RR, 3) : 0;
  static constexpr int S_DD = TUNED ? tuned_layout(D, Q, DIFF, ES, RR, 0) : odd_pad(D2);
  static constexpr int S_QD = TUNED ? tuned_layout(D, Q, DIFF, ES, RR, 1) : odd_pad(QD);
  static constexpr int S_QQ = TUNED ? tuned_layout(D, Q, DIFF, ES, RR, 2) : odd_pad(Q2);
  static constexpr int NC_FWD = DIFF ? 2 : 1;  // arrays after the x phase (B x, G x)
  static constexpr int NC_Q = DIFF ? 3 : 1;    // arrays at quadrature points
  // buffer A: E0 [i][line], T2 [c][k][line], S5 [c][qx][line]
  static constexpr int SZ_A_MIN = cmax(D * S_DD, cmax(NC_Q * D * S_QQ, NC_FWD * Q * S_DD));
  // buffer B: T1 [c][j][line], S4 [c][qy][line], Ye [a]
  static constexpr int SZ_B_MIN = cmax(NC_FWD * D * S_QD, cmax(NC_Q * Q * S_QD, D3));
  static constexpr int SZ_A = TUNED ? TUNED : SZ_A_MIN;
  static constexpr int SZ_B = TUNED ? tuned_layout(D, Q, DIFF, ES, RR, 4) : SZ_B_MIN;
  static_assert(S_DD >= D2 && S_QD >= QD && S_QQ >= Q2 && SZ_A >= SZ_A_MIN && SZ_B >= SZ_B_MIN,
                "shared-memory layout too small");
  static constexpr int PER_ELEM = SZ_A + SZ_B;
};

// DIFF: diffusion (qdata [e][qz][6][qy][qx]: xx, xy, xz, yy, yz, zz) or mass ([e][qz][qy][qx]).
// VT: element type of the x and y vectors (double; float for the FP32 inner solves).
// MULTI: several right-hand sides per launch (nrhs); when false the launch handles exactly one.
//
// One thread block's share of the fused apply: elements [blk NE, blk NE + NE) of the element list
// (fewer at its end), for the right-hand sides.  Returns the thread's partial of x^T A x when
// want_dot (single right-hand side).  smem_raw holds the NE elements' buffers, wexp NT / 32 ints
// of shared memory.  Used by the per-order kernel (blk = blockIdx.x) and by the persistent
// multi-order kernel (blk = the work item's block within its order group).
template <int D, int Q, int NE, int NT, bool DIFF, class Ar, bool REREAD, class VT, bool MULTI>
__device__ __forceinline__ typename Ar::DotAcc pa_apply_block(
    const int32_t* __restrict__ map, const typename Ar::QdT* __restrict__ qd,
    const int32_t* __restrict__ qscale, int qshift, const VT* __restrict__ x0,
    VT* __restrict__ y0, int64_t ne, int64_t blk, bool want_dot, int nrhs, int64_t ldx,
    int64_t ldy, const typename Ar::template Tab<D, Q>& tab, unsigned char* smem_raw,
    int* wexp) {
  using T = typename Ar::T;
  using L = ApplyLayout<D, Q, DIFF, (int)sizeof(T), REREAD>;
  constexpr int D2 = L::D2, D3 = L::D3, Q2 = L::Q2, QD = L::QD;
  constexpr int S_DD = L::S_DD, S_QD = L::S_QD, S_QQ = L::S_QQ;
  constexpr int SZ_A = L::SZ_A, SZ_B = L::SZ_B;
  constexpr int NQD = DIFF ? 6 : 1;
  constexpr bool PREFETCH_QD = Ar::kPrefetchQd;

  T* bufA = reinterpret_cast<T*>(smem_raw);
  T* bufB = bufA + NE * SZ_A;

  const int64_t e0 = blk * NE;
  const int nel = (int)((ne - e0) < NE ? (ne - e0) : NE);
  const int tid = threadIdx.x;
  auto dacc = Ar::dot_zero();

  // Several right-hand sides (x0 + r ldx -> y0 + r ldy) are applied one after the other by the
  // same block: after the first, the block's dof map and quadrature data come from L2.
  // The block's quadrature data (contiguous: elements e0 .. e0 + nel - 1) are first needed in the
  // z phase; a bulk prefetch into L2 issued now lets them arrive during the gather and the x and
  // y phases instead of stalling the z phase's loads on HBM latency.
  if (PREFETCH_QD && tid < 32) {
    constexpr int64_t QD_BYTES = (int64_t)NQD * Q * Q2 * sizeof(typename Ar::QdT);
    constexpr int64_t CHUNK = 32 * 1024;
    // the block's byte range rounded inward to 16-byte boundaries (the bulk operations' unit),
    // so that it stays inside the array
    const uintptr_t lo = (reinterpret_cast<uintptr_t>(qd) + e0 * QD_BYTES + 15) & ~(uintptr_t)15;
    const uintptr_t hi = (reinterpret_cast<uintptr_t>(qd) + (e0 + nel) * QD_BYTES) & ~(uintptr_t)15;
    for (uintptr_t a = lo + (uintptr_t)tid * CHUNK; a < hi; a += 32 * CHUNK) {
      const uint32_t n = (uint32_t)((hi - a) < (uintptr_t)CHUNK ? (hi - a) : (uintptr_t)CHUNK);
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"(n) : "memory");
    }
  }

  const int nr = MULTI ? nrhs : 1;
  for (int rhs = 0; rhs < nr; ++rhs) {
  const VT* __restrict__ x = x0 + rhs * ldx;
  VT* __restrict__ y = y0 + rhs * ldy;
  if (rhs > 0) __syncthreads();  // the previous scatter has read its last bufB value

  // ---- gather (G): E0[i][j*D + k] = x[map[e][i + D j + D^2 k]].  Scaled policies keep the
  //      FP64 value in the slot (same 8 bytes) and note its exponent; the x phase converts it
  //      with the block's scale 2^(1023 - largest exponent).
  //      Two stages per chunk of GCH items, so that every thread has its independent loads in
  //      flight at once: the block's dof-map entries (contiguous: item t = el D^3 + a), then the
  //      values.  The chunk bounds the registers the staging takes.
  constexpr int GPT = (NE * D3 + NT - 1) / NT;  // gather items per thread
  constexpr int GCH = GPT < 8 ? GPT : 8;
  const int ntot = nel * D3;
  const int32_t* __restrict__ mb = map + e0 * D3;
  {
    int emax = 0;
#pragma unroll 1
    for (int u0 = 0; u0 < GPT; u0 += GCH) {
      int32_t gi[GCH];
#pragma unroll
      for (int u = 0; u < GCH; ++u) {
        const int t = tid + (u0 + u) * NT;
        gi[u] = t < ntot ? __ldg(&mb[t]) : 0;
      }
      VT xv[GCH];
#pragma unroll
      for (int u = 0; u < GCH; ++u) {
        const int t = tid + (u0 + u) * NT;
        xv[u] = t < ntot ? __ldg(&x[gi[u]]) : VT(0);
      }
#pragma unroll
      for (int u = 0; u < GCH; ++u) {
        const int t = tid + (u0 + u) * NT;
        if (t < ntot) {
          const int el = t / D3, a = t - el * D3;
          const int i = a % D, j = (a / D) % D, k = a / D2;
          if constexpr (Ar::kScaled) {
            reinterpret_cast<double*>(bufA)[el * SZ_A + i * S_DD + j * D + k] = xv[u];
            emax = max(emax, f64_exponent(xv[u]));
          } else {
            bufA[el * SZ_A + i * S_DD + j * D + k] = Ar::from_vec(xv[u]);
          }
        }
      }
    }
    if constexpr (Ar::kScaled) {
      emax = __reduce_max_sync(0xffffffffu, emax);
      if ((tid & 31) == 0) wexp[tid >> 5] = emax;
    }
  }
  __syncthreads();
  int xexp = 1023;  // biased exponent that the scaled inputs map to 2^0
  if constexpr (Ar::kScaled) {
    xexp = 0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) xexp = max(xexp, wexp[w]);
  }

  // ---- x phase: contract i -> qx.  line (j, k); out T1c[j][k*Q + qx], c = (B x, G x)
  if constexpr (Ar::kEvenOdd) {
    eo::x_phase<D, Q, NT, DIFF, L, Ar>(tab, bufA, bufB, nel, tid, xexp);
  } else {
    for (int t = tid; t < nel * D2; t += NT) {
      const int el = t / D2, l = t - el * D2;
      const int j = l / D, k = l - j * D;
      const T* in = bufA + el * SZ_A + l;
      T v[D];
      float m = 0.0f;
  #pragma unroll
      for (int i = 0; i < D; ++i) {
        if constexpr (Ar::kScaled)
          v[i] = Ar::from_raw(reinterpret_cast<const double*>(in)[i * S_DD], 1023 - xexp);
        else
          v[i] = in[i * S_DD];
        m = Ar::amax(m, v[i]);
      }
      const auto sb = Ar::sigB(tab, m, false);
      T* outb = bufB + el * SZ_B + j * S_QD + k * Q;
  #pragma unroll
      for (int qx = 0; qx < Q; ++qx) {
        auto ab = Ar::begin(sb);
  #pragma unroll
        for (int i = 0; i < D; ++i) Ar::amadB(ab, tab, qx, i, v[i]);
        outb[qx] = Ar::end(ab, sb);
      }
      if constexpr (DIFF) {
        const auto sg = Ar::sigG(tab, m, false);
  #pragma unroll
        for (int qx = 0; qx < Q; ++qx) {
          auto ag = Ar::begin(sg);
  #pragma unroll
          for (int i = 0; i < D; ++i) Ar::amadG(ag, tab, qx, i, v[i]);
          outb[D * S_QD + qx] = Ar::end(ag, sg);
        }
      }
    }
  }
  __syncthreads();

  // ---- y phase: contract j -> qy.  line (k, qx); out T2c[k][qy*Q + qx]
  //      diffusion: c0 = B_y (G_x x), c1 = G_y (B_x x), c2 = B_y (B_x x)
  if constexpr (Ar::kEvenOdd) {
    eo::y_phase<D, Q, NT, DIFF, L, Ar>(tab, bufB, bufA, nel, tid);
  } else {
    for (int t = tid; t < nel * QD; t += NT) {
      const int el = t / QD, l = t - el * QD;
      const int k = l / Q, qx = l - k * Q;
      const T* in = bufB + el * SZ_B + l;
      T vb[D];
      float mb = 0.0f;
  #pragma unroll
      for (int j = 0; j < D; ++j) {
        vb[j] = in[j * S_QD];
        mb = Ar::amax(mb, vb[j]);
      }
      T* out = bufA + el * SZ_A + k * S_QQ + qx;
      const auto s_bb = Ar::sigB(tab, mb, false);
      if constexpr (DIFF) {
        T vg[D];
        float mg = 0.0f;
  #pragma unroll
        for (int j = 0; j < D; ++j) {
          vg[j] = in[D * S_QD + j * S_QD];
          mg = Ar::amax(mg, vg[j]);
        }
        const auto s_bg = Ar::sigB(tab, mg, false), s_gb = Ar::sigG(tab, mb, false);
  #pragma unroll
        for (int qy = 0; qy < Q; ++qy) {
          auto a0 = Ar::begin(s_bg), a1 = Ar::begin(s_gb), a2 = Ar::begin(s_bb);
  #pragma unroll
          for (int j = 0; j < D; ++j) {
            Ar::amadB(a0, tab, qy, j, vg[j]);
            Ar::amadG(a1, tab, qy, j, vb[j]);
            Ar::amadB(a2, tab, qy, j, vb[j]);
          }
          out[qy * Q] = Ar::end(a0, s_bg);
          out[D * S_QQ + qy * Q] = Ar::end(a1, s_gb);
          out[2 * D * S_QQ + qy * Q] = Ar::end(a2, s_bb);
        }
      } else {
  #pragma unroll
        for (int qy = 0; qy < Q; ++qy) {
          auto a0 = Ar::begin(s_bb);
  #pragma unroll
          for (int j = 0; j < D; ++j) Ar::amadB(a0, tab, qy, j, vb[j]);
          out[qy * Q] = Ar::end(a0, s_bb);
        }
      }
    }
  }
  __syncthreads();

  // ---- z phase: contract k -> qz, apply D, contract qz -> k.  line (qy, qx)
  //      out S4c[qy][k*Q + qx].  The forward contraction is anchored (bound from the inputs),
  //      the pointwise product too (exact bound per point); the transposed contraction, whose
  //      inputs appear only inside the qz loop, is anchored in a second pass over the column
  //      for Q <= 6 and compensated otherwise.
  if constexpr (Ar::kEvenOdd) {
    eo::z_phase<D, Q, NT, DIFF, L, Ar>(tab, bufA, bufB, qd, e0, nel, tid);
  } else {
    for (int t = tid; t < nel * Q2; t += NT) {
      const int el = t / Q2, l = t - el * Q2;
      const int qy = l / Q, qx = l - qy * Q;
      const T* in = bufA + el * SZ_A + l;
      const typename Ar::QdT* qe = qd + (e0 + el) * (int64_t)(NQD * Q * Q2) + l;
      T* out = bufB + el * SZ_B + qy * S_QD + qx;
      if constexpr (DIFF) {
        // bounds of the three input columns (one pass over shared memory)
        float m0 = 0.0f, m1 = 0.0f, m2 = 0.0f;
  #pragma unroll
        for (int k = 0; k < D; ++k) {
          m0 = Ar::amax(m0, in[k * S_QQ]);
          m1 = Ar::amax(m1, in[D * S_QQ + k * S_QQ]);
          m2 = Ar::amax(m2, in[2 * D * S_QQ + k * S_QQ]);
        }
        const auto s0 = Ar::sigB(tab, m0, false), s1 = Ar::sigB(tab, m1, false);
        const auto s2 = Ar::sigG(tab, m2, false);
        // Inputs are re-read from shared memory at every qz when REREAD (the empty asm with a
        // memory clobber keeps the compiler from caching them in registers): only the 3D
        // accumulators stay live, which keeps high orders at two or more blocks per SM.
        // ZTWO (float-float, Q <= 6): keep the column's v values and finish with an anchored
        // transposed contraction; otherwise accumulate w with compensated steps inside the loop
        constexpr bool ZTWO = Ar::kAnchored && Q <= 6;
        constexpr int NW_ = ZTWO ? 1 : D;
        constexpr int NV_ = ZTWO ? Q : 1;
        T w0[NW_], w1[NW_], w2[NW_];
        T vs0[NV_], vs1[NV_], vs2[NV_];
        float vm0 = 0.0f, vm1 = 0.0f, vm2 = 0.0f;
  #pragma unroll
        for (int k = 0; k < NW_; ++k) w0[k] = w1[k] = w2[k] = Ar::zero();
        // quadrature data of the next qz is loaded one iteration ahead (register double buffer)
        T nd[6];
  #pragma unroll
        for (int c = 0; c < 6; ++c) nd[c] = Ar::load_qd(qe + c * Q2);
  #pragma unroll
        for (int qz = 0; qz < Q; ++qz) {
          if constexpr (REREAD) asm volatile("" ::: "memory");
          T cd[6];
  #pragma unroll
          for (int c = 0; c < 6; ++c) cd[c] = nd[c];
          if (qz + 1 < Q) {
  #pragma unroll
            for (int c = 0; c < 6; ++c) nd[c] = Ar::load_qd(qe + ((qz + 1) * 6 + c) * Q2);
          }
          auto a0 = Ar::begin(s0), a1 = Ar::begin(s1), a2 = Ar::begin(s2);
  #pragma unroll
          for (int k = 0; k < D; ++k) {
            Ar::amadB(a0, tab, qz, k, in[k * S_QQ]);
            Ar::amadB(a1, tab, qz, k, in[D * S_QQ + k * S_QQ]);
            Ar::amadG(a2, tab, qz, k, in[2 * D * S_QQ + k * S_QQ]);
          }
          const T g0 = Ar::end(a0, s0), g1 = Ar::end(a1, s1), g2 = Ar::end(a2, s2);
          // v = D g, D symmetric: (xx, xy, xz, yy, yz, zz)
          const T v0 = Ar::dot3(cd[0], g0, cd[1], g1, cd[2], g2);
          const T v1 = Ar::dot3(cd[1], g0, cd[3], g1, cd[4], g2);
          const T v2 = Ar::dot3(cd[2], g0, cd[4], g1, cd[5], g2);
          if constexpr (ZTWO) {
            vs0[qz] = v0;
            vs1[qz] = v1;
            vs2[qz] = v2;
            vm0 = Ar::amax(vm0, v0);
            vm1 = Ar::amax(vm1, v1);
            vm2 = Ar::amax(vm2, v2);
          } else {
  #pragma unroll
            for (int k = 0; k < D; ++k) {
              Ar::madB(w0[k], tab, qz, k, v0);
              Ar::madB(w1[k], tab, qz, k, v1);
              Ar::madG(w2[k], tab, qz, k, v2);
            }
          }
        }
        if constexpr (ZTWO) {
          // second pass over the column: the transposed z contraction, anchored now that the
          // bounds max_qz |v_c| are known
          const auto t0 = Ar::sigB(tab, vm0, true), t1 = Ar::sigB(tab, vm1, true);
          const auto t2 = Ar::sigG(tab, vm2, true);
  #pragma unroll
          for (int k = 0; k < D; ++k) {
            auto r0 = Ar::begin(t0), r1 = Ar::begin(t1), r2 = Ar::begin(t2);
  #pragma unroll
            for (int qz = 0; qz < Q; ++qz) {
              Ar::amadB(r0, tab, qz, k, vs0[qz]);
              Ar::amadB(r1, tab, qz, k, vs1[qz]);
              Ar::amadG(r2, tab, qz, k, vs2[qz]);
            }
            out[k * Q] = Ar::end(r0, t0);
            out[Q * S_QD + k * Q] = Ar::end(r1, t1);
            out[2 * Q * S_QD + k * Q] = Ar::end(r2, t2);
          }
        } else {
  #pragma unroll
          for (int k = 0; k < D; ++k) {
            out[k * Q] = Ar::norm(w0[k]);
            out[Q * S_QD + k * Q] = Ar::norm(w1[k]);
            out[2 * Q * S_QD + k * Q] = Ar::norm(w2[k]);
          }
        }
      } else {
        float m = 0.0f;
  #pragma unroll
        for (int k = 0; k < D; ++k) m = Ar::amax(m, in[k * S_QQ]);
        const auto s = Ar::sigB(tab, m, false);
        T w[D];
  #pragma unroll
        for (int k = 0; k < D; ++k) w[k] = Ar::zero();
        T nd = Ar::load_qd(qe);
  #pragma unroll
        for (int qz = 0; qz < Q; ++qz) {
          if constexpr (REREAD) asm volatile("" ::: "memory");
          const T cd = nd;
          if (qz + 1 < Q) nd = Ar::load_qd(qe + (qz + 1) * Q2);
          auto a = Ar::begin(s);
  #pragma unroll
          for (int k = 0; k < D; ++k) Ar::amadB(a, tab, qz, k, in[k * S_QQ]);
          const T v = Ar::norm(Ar::mul(cd, Ar::end(a, s)));
  #pragma unroll
          for (int k = 0; k < D; ++k) Ar::madB(w[k], tab, qz, k, v);
        }
  #pragma unroll
        for (int k = 0; k < D; ++k) out[k * Q] = Ar::norm(w[k]);
      }
    }
  }
  __syncthreads();

  // ---- y^T phase: contract qy -> j.  line (k, qx); out S5c[qx][j*D + k]
  //      diffusion: c0 (-> G_x^T) = B_y^T s0, c1 (-> B_x^T) = G_y^T s1 + B_y^T s2
  //      (outer-product form over qy with anchored accumulators; bounds from a first pass)
  if constexpr (Ar::kEvenOdd) {
    eo::yt_phase<D, Q, NT, DIFF, L, Ar>(tab, bufB, bufA, nel, tid);
  } else {
    for (int t = tid; t < nel * QD; t += NT) {
      const int el = t / QD, l = t - el * QD;
      const int k = l / Q, qx = l - k * Q;
      const T* in = bufB + el * SZ_B + l;
      T* out = bufA + el * SZ_A + qx * S_DD + k;
      if constexpr (DIFF) {
        float m0 = 0.0f, m1 = 0.0f, m2 = 0.0f;
  #pragma unroll
        for (int qy = 0; qy < Q; ++qy) {
          m0 = Ar::amax(m0, in[qy * S_QD]);
          m1 = Ar::amax(m1, in[Q * S_QD + qy * S_QD]);
          m2 = Ar::amax(m2, in[2 * Q * S_QD + qy * S_QD]);
        }
        const auto sg = Ar::sigB(tab, m0, true), sb = Ar::sigGB(tab, m1, m2, true);
        typename Ar::Acc rg[D], rb[D];
  #pragma unroll
        for (int j = 0; j < D; ++j) {
          rg[j] = Ar::begin(sg);
          rb[j] = Ar::begin(sb);
        }
  #pragma unroll
        for (int qy = 0; qy < Q; ++qy) {
          const T a0 = in[qy * S_QD], a1 = in[Q * S_QD + qy * S_QD], a2 = in[2 * Q * S_QD + qy * S_QD];
  #pragma unroll
          for (int j = 0; j < D; ++j) {
            Ar::amadB(rg[j], tab, qy, j, a0);
            Ar::amadG(rb[j], tab, qy, j, a1);
            Ar::amadB(rb[j], tab, qy, j, a2);
          }
        }
  #pragma unroll
        for (int j = 0; j < D; ++j) {
          out[j * D] = Ar::end(rg[j], sg);
          out[Q * S_DD + j * D] = Ar::end(rb[j], sb);
        }
      } else {
        float m0 = 0.0f;
  #pragma unroll
        for (int qy = 0; qy < Q; ++qy) m0 = Ar::amax(m0, in[qy * S_QD]);
        const auto s0 = Ar::sigB(tab, m0, true);
        typename Ar::Acc r[D];
  #pragma unroll
        for (int j = 0; j < D; ++j) r[j] = Ar::begin(s0);
  #pragma unroll
        for (int qy = 0; qy < Q; ++qy) {
          const T a0 = in[qy * S_QD];
  #pragma unroll
          for (int j = 0; j < D; ++j) Ar::amadB(r[j], tab, qy, j, a0);
        }
  #pragma unroll
        for (int j = 0; j < D; ++j) out[j * D] = Ar::end(r[j], s0);
      }
    }
  }
  __syncthreads();

  // ---- x^T phase: contract qx -> i.  line (j, k); out Ye[i + D j + D^2 k]
  if constexpr (Ar::kEvenOdd) {
    eo::xt_phase<D, Q, NT, DIFF, L, Ar>(tab, bufA, bufB, nel, tid);
  } else {
    for (int t = tid; t < nel * D2; t += NT) {
      const int el = t / D2, l = t - el * D2;
      const int j = l / D, k = l - j * D;
      const T* in = bufA + el * SZ_A + l;
      float mg = 0.0f, mb = 0.0f;
  #pragma unroll
      for (int qx = 0; qx < Q; ++qx) {
        mg = Ar::amax(mg, in[qx * S_DD]);
        if constexpr (DIFF) mb = Ar::amax(mb, in[Q * S_DD + qx * S_DD]);
      }
      const auto s = DIFF ? Ar::sigGB(tab, mg, mb, true) : Ar::sigB(tab, mg, true);
      typename Ar::Acc r[D];
  #pragma unroll
      for (int i = 0; i < D; ++i) r[i] = Ar::begin(s);
  #pragma unroll
      for (int qx = 0; qx < Q; ++qx) {
        const T ag = in[qx * S_DD];
        if constexpr (DIFF) {
          const T ab = in[Q * S_DD + qx * S_DD];
  #pragma unroll
          for (int i = 0; i < D; ++i) {
            Ar::amadG(r[i], tab, qx, i, ag);
            Ar::amadB(r[i], tab, qx, i, ab);
          }
        } else {
  #pragma unroll
          for (int i = 0; i < D; ++i) Ar::amadB(r[i], tab, qx, i, ag);
        }
      }
      T* out = bufB + el * SZ_B + j * D + k * D2;
  #pragma unroll
      for (int i = 0; i < D; ++i) out[i] = Ar::end(r[i], s);
    }
  }
  __syncthreads();

  // ---- scatter-add (G^T); optionally the block's share of x^T A x = sum_e x_e . (A_e x_e),
  //      accumulated from the FP64 inputs and the FP64 results that are scattered
  //      (the map entries of a chunk first, as in the gather)
#pragma unroll 1
  for (int u0 = 0; u0 < GPT; u0 += GCH) {
    int32_t gs[GCH];
#pragma unroll
    for (int u = 0; u < GCH; ++u) {
      const int t = tid + (u0 + u) * NT;
      gs[u] = t < ntot ? __ldg(&mb[t]) : 0;
    }
#pragma unroll
    for (int u = 0; u < GCH; ++u) {
      const int t = tid + (u0 + u) * NT;
      if (t >= ntot) continue;
      const int el = t / D3, a = t - el * D3;
      const int32_t g = gs[u];
      const T v = bufB[el * SZ_B + a];
      if constexpr (std::is_same<VT, float>::value) {
        Ar::scatter(&y[g], v);
        if (want_dot) Ar::dot_acc(dacc, __ldg(&x[g]), v);
      } else {
        // scaled policies: undo the input scale and the element's quadrature-data scale; FP32
        // data: undo its global shift
        const int off = Ar::kScaled ? (xexp - 1023) + __ldg(&qscale[e0 + el]) : qshift;
        const double vd = Ar::widen(v, off);
        atomicAdd(&y[g], vd);
        if (want_dot) Ar::dot_acc(dacc, __ldg(&x[g]), vd);
      }
    }
  }
  }  // right-hand sides
  return dacc;
}

// The per-order fused apply: block b applies elements [b NE, b NE + NE).
template <int D, int Q, int NE, int NT, bool DIFF, class Ar, bool REREAD, int MINB, class VT,
          bool MULTI>
__global__ void __launch_bounds__(NT, MINB) k_pa_apply(const int32_t* __restrict__ map,
                                                 const typename Ar::QdT* __restrict__ qd,
                                                 const int32_t* __restrict__ qscale,
                                                 int qshift, const VT* __restrict__ x0,
                                                 VT* __restrict__ y0, int64_t ne,
                                                 const int* __restrict__ skip,
                                                 double* __restrict__ dot_part, int nrhs,
                                                 int64_t ldx, int64_t ldy,
                                                 const typename Ar::template Tab<D, Q> tab) {
  // optional device flag: a nonzero value turns the launch into a no-op (used by the CG loop
  // once it has converged, so that already-queued iterations cost nothing)
  if (skip != nullptr && *skip != 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int wexp[NT / 32];  // scaled policies: per-warp largest input exponent
  const int tid = threadIdx.x;
  auto dacc = pa_apply_block<D, Q, NE, NT, DIFF, Ar, REREAD, VT, MULTI>(
      map, qd, qscale, qshift, x0, y0, ne, blockIdx.x, dot_part != nullptr, nrhs, ldx, ldy, tab,
      smem_raw, wexp);
  if (dot_part != nullptr) {  // (single right-hand side only)  // deterministic block reduction (fixed shuffle tree, warp order)
    double dsum = Ar::dot_value(dacc);
    __shared__ double wsum[NT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_down_sync(0xffffffffu, dsum, o);
    if ((tid & 31) == 0) wsum[tid >> 5] = dsum;
    __syncthreads();
    if (tid == 0) {
      double tot = 0.0;
#pragma unroll
      for (int w = 0; w < NT / 32; ++w) tot += wsum[w];
      dot_part[blockIdx.x] = tot;
    }
  }
}

}  // namespace fe
