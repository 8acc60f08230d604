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
// Shared-memory arrays are stored "summed index slowest" with every slab padded to an odd
// number of 8-byte words, so both unit-stride and slab-stride accesses are free of bank
// conflicts (the concern of Sections III-C/D, solved by layout rather than fragment maps).
// The z-direction phase fuses the forward z contraction, the pointwise D and the transposed z
// contraction in registers, one (qx, qy) column per thread.
#pragma once

#include "fe_arith.cuh"

namespace fe {

__host__ __device__ constexpr int odd_pad(int n) { return (n % 2 == 0) ? n + 1 : n; }
__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }

template <int D, int Q, bool DIFF>
struct ApplyLayout {
  static constexpr int D2 = D * D, D3 = D * D * D, Q2 = Q * Q, QD = Q * D;
  static constexpr int S_DD = odd_pad(D2), S_QD = odd_pad(QD), S_QQ = odd_pad(Q2);
  static constexpr int NC_FWD = DIFF ? 2 : 1;  // arrays after the x phase (B x, G x)
  static constexpr int NC_Q = DIFF ? 3 : 1;    // arrays at quadrature points
  // buffer A: E0 [i][line], T2 [c][k][line], S5 [c][qx][line]
  static constexpr int SZ_A = cmax(D * S_DD, cmax(NC_Q * D * S_QQ, NC_FWD * Q * S_DD));
  // buffer B: T1 [c][j][line], S4 [c][qy][line], Ye [a]
  static constexpr int SZ_B = cmax(NC_FWD * D * S_QD, cmax(NC_Q * Q * S_QD, D3));
  static constexpr int PER_ELEM = SZ_A + SZ_B;
};

// DIFF: diffusion (qdata [e][qz][6][qy][qx]: xx, xy, xz, yy, yz, zz) or mass ([e][qz][qy][qx]).
template <int D, int Q, int NE, int NT, bool DIFF, class Ar>
__global__ void __launch_bounds__(NT) k_pa_apply(const int32_t* __restrict__ map,
                                                 const double* __restrict__ qd,
                                                 const double* __restrict__ x,
                                                 double* __restrict__ y, int64_t ne,
                                                 const int* __restrict__ skip,
                                                 const typename Ar::template Tab<D, Q> tab) {
  using T = typename Ar::T;
  using L = ApplyLayout<D, Q, DIFF>;
  constexpr int D2 = L::D2, D3 = L::D3, Q2 = L::Q2, QD = L::QD;
  constexpr int S_DD = L::S_DD, S_QD = L::S_QD, S_QQ = L::S_QQ;
  constexpr int SZ_A = L::SZ_A, SZ_B = L::SZ_B;
  constexpr int NQD = DIFF ? 6 : 1;

  // optional device flag: a nonzero value turns the launch into a no-op (used by the CG loop
  // once it has converged, so that already-queued iterations cost nothing)
  if (skip != nullptr && *skip != 0) return;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* bufA = reinterpret_cast<T*>(smem_raw);
  T* bufB = bufA + NE * SZ_A;

  const int64_t e0 = (int64_t)blockIdx.x * NE;
  const int nel = (int)((ne - e0) < NE ? (ne - e0) : NE);
  const int tid = threadIdx.x;

  // ---- gather (G): E0[i][j*D + k] = x[map[e][i + D j + D^2 k]]
  for (int t = tid; t < nel * D3; t += NT) {
    const int el = t / D3, a = t - el * D3;
    const int i = a % D, j = (a / D) % D, k = a / D2;
    const int32_t g = __ldg(&map[(e0 + el) * D3 + a]);
    bufA[el * SZ_A + i * S_DD + j * D + k] = Ar::from_f64(__ldg(&x[g]));
  }
  __syncthreads();

  // ---- x phase: contract i -> qx.  line (j, k); out T1c[j][k*Q + qx], c = (B x, G x)
  for (int t = tid; t < nel * D2; t += NT) {
    const int el = t / D2, l = t - el * D2;
    const int j = l / D, k = l - j * D;
    const T* in = bufA + el * SZ_A + l;
    T v[D];
#pragma unroll
    for (int i = 0; i < D; ++i) v[i] = in[i * S_DD];
    T* outb = bufB + el * SZ_B + j * S_QD + k * Q;
#pragma unroll
    for (int qx = 0; qx < Q; ++qx) {
      T ab = Ar::zero();
#pragma unroll
      for (int i = 0; i < D; ++i) Ar::madB(ab, tab, qx, i, v[i]);
      outb[qx] = Ar::norm(ab);
      if constexpr (DIFF) {
        T ag = Ar::zero();
#pragma unroll
        for (int i = 0; i < D; ++i) Ar::madG(ag, tab, qx, i, v[i]);
        outb[D * S_QD + qx] = Ar::norm(ag);
      }
    }
  }
  __syncthreads();

  // ---- y phase: contract j -> qy.  line (k, qx); out T2c[k][qy*Q + qx]
  //      diffusion: c0 = B_y (G_x x), c1 = G_y (B_x x), c2 = B_y (B_x x)
  for (int t = tid; t < nel * QD; t += NT) {
    const int el = t / QD, l = t - el * QD;
    const int k = l / Q, qx = l - k * Q;
    const T* in = bufB + el * SZ_B + l;
    T vb[D];
#pragma unroll
    for (int j = 0; j < D; ++j) vb[j] = in[j * S_QD];
    T* out = bufA + el * SZ_A + k * S_QQ + qx;
    if constexpr (DIFF) {
      T vg[D];
#pragma unroll
      for (int j = 0; j < D; ++j) vg[j] = in[D * S_QD + j * S_QD];
#pragma unroll
      for (int qy = 0; qy < Q; ++qy) {
        T a0 = Ar::zero(), a1 = Ar::zero(), a2 = Ar::zero();
#pragma unroll
        for (int j = 0; j < D; ++j) {
          Ar::madB(a0, tab, qy, j, vg[j]);
          Ar::madG(a1, tab, qy, j, vb[j]);
          Ar::madB(a2, tab, qy, j, vb[j]);
        }
        out[qy * Q] = Ar::norm(a0);
        out[D * S_QQ + qy * Q] = Ar::norm(a1);
        out[2 * D * S_QQ + qy * Q] = Ar::norm(a2);
      }
    } else {
#pragma unroll
      for (int qy = 0; qy < Q; ++qy) {
        T a0 = Ar::zero();
#pragma unroll
        for (int j = 0; j < D; ++j) Ar::madB(a0, tab, qy, j, vb[j]);
        out[qy * Q] = Ar::norm(a0);
      }
    }
  }
  __syncthreads();

  // ---- z phase: contract k -> qz, apply D, contract qz -> k.  line (qy, qx)
  //      out S4c[qy][k*Q + qx]
  for (int t = tid; t < nel * Q2; t += NT) {
    const int el = t / Q2, l = t - el * Q2;
    const int qy = l / Q, qx = l - qy * Q;
    const T* in = bufA + el * SZ_A + l;
    const double* qe = qd + (e0 + el) * (int64_t)(NQD * Q * Q2) + l;
    T* out = bufB + el * SZ_B + qy * S_QD + qx;
    if constexpr (DIFF) {
      T u0[D], u1[D], u2[D], w0[D], w1[D], w2[D];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        u0[k] = in[k * S_QQ];
        u1[k] = in[D * S_QQ + k * S_QQ];
        u2[k] = in[2 * D * S_QQ + k * S_QQ];
        w0[k] = w1[k] = w2[k] = Ar::zero();
      }
#pragma unroll
      for (int qz = 0; qz < Q; ++qz) {
        T g0 = Ar::zero(), g1 = Ar::zero(), g2 = Ar::zero();
#pragma unroll
        for (int k = 0; k < D; ++k) {
          Ar::madB(g0, tab, qz, k, u0[k]);
          Ar::madB(g1, tab, qz, k, u1[k]);
          Ar::madG(g2, tab, qz, k, u2[k]);
        }
        g0 = Ar::norm(g0);
        g1 = Ar::norm(g1);
        g2 = Ar::norm(g2);
        const double* qq = qe + qz * 6 * Q2;
        const T dxx = Ar::load_qd(qq), dxy = Ar::load_qd(qq + Q2), dxz = Ar::load_qd(qq + 2 * Q2);
        const T dyy = Ar::load_qd(qq + 3 * Q2), dyz = Ar::load_qd(qq + 4 * Q2);
        const T dzz = Ar::load_qd(qq + 5 * Q2);
        T v0 = Ar::mul(dxx, g0), v1 = Ar::mul(dxy, g0), v2 = Ar::mul(dxz, g0);
        Ar::mad(v0, dxy, g1);
        Ar::mad(v0, dxz, g2);
        Ar::mad(v1, dyy, g1);
        Ar::mad(v1, dyz, g2);
        Ar::mad(v2, dyz, g1);
        Ar::mad(v2, dzz, g2);
        v0 = Ar::norm(v0);
        v1 = Ar::norm(v1);
        v2 = Ar::norm(v2);
#pragma unroll
        for (int k = 0; k < D; ++k) {
          Ar::madB(w0[k], tab, qz, k, v0);
          Ar::madB(w1[k], tab, qz, k, v1);
          Ar::madG(w2[k], tab, qz, k, v2);
        }
      }
#pragma unroll
      for (int k = 0; k < D; ++k) {
        out[k * Q] = Ar::norm(w0[k]);
        out[Q * S_QD + k * Q] = Ar::norm(w1[k]);
        out[2 * Q * S_QD + k * Q] = Ar::norm(w2[k]);
      }
    } else {
      T u[D], w[D];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        u[k] = in[k * S_QQ];
        w[k] = Ar::zero();
      }
#pragma unroll
      for (int qz = 0; qz < Q; ++qz) {
        T g = Ar::zero();
#pragma unroll
        for (int k = 0; k < D; ++k) Ar::madB(g, tab, qz, k, u[k]);
        const T v = Ar::norm(Ar::mul(Ar::load_qd(qe + qz * Q2), Ar::norm(g)));
#pragma unroll
        for (int k = 0; k < D; ++k) Ar::madB(w[k], tab, qz, k, v);
      }
#pragma unroll
      for (int k = 0; k < D; ++k) out[k * Q] = Ar::norm(w[k]);
    }
  }
  __syncthreads();

  // ---- y^T phase: contract qy -> j.  line (k, qx); out S5c[qx][j*D + k]
  //      diffusion: c0 (-> G_x^T) = B_y^T s0, c1 (-> B_x^T) = G_y^T s1 + B_y^T s2
  for (int t = tid; t < nel * QD; t += NT) {
    const int el = t / QD, l = t - el * QD;
    const int k = l / Q, qx = l - k * Q;
    const T* in = bufB + el * SZ_B + l;
    T* out = bufA + el * SZ_A + qx * S_DD + k;
    if constexpr (DIFF) {
      T s0[Q], s1[Q], s2[Q];
#pragma unroll
      for (int qy = 0; qy < Q; ++qy) {
        s0[qy] = in[qy * S_QD];
        s1[qy] = in[Q * S_QD + qy * S_QD];
        s2[qy] = in[2 * Q * S_QD + qy * S_QD];
      }
#pragma unroll
      for (int j = 0; j < D; ++j) {
        T rg = Ar::zero(), rb = Ar::zero();
#pragma unroll
        for (int qy = 0; qy < Q; ++qy) {
          Ar::madB(rg, tab, qy, j, s0[qy]);
          Ar::madG(rb, tab, qy, j, s1[qy]);
          Ar::madB(rb, tab, qy, j, s2[qy]);
        }
        out[j * D] = Ar::norm(rg);
        out[Q * S_DD + j * D] = Ar::norm(rb);
      }
    } else {
      T s0[Q];
#pragma unroll
      for (int qy = 0; qy < Q; ++qy) s0[qy] = in[qy * S_QD];
#pragma unroll
      for (int j = 0; j < D; ++j) {
        T r = Ar::zero();
#pragma unroll
        for (int qy = 0; qy < Q; ++qy) Ar::madB(r, tab, qy, j, s0[qy]);
        out[j * D] = Ar::norm(r);
      }
    }
  }
  __syncthreads();

  // ---- x^T phase: contract qx -> i.  line (j, k); out Ye[i + D j + D^2 k]
  for (int t = tid; t < nel * D2; t += NT) {
    const int el = t / D2, l = t - el * D2;
    const int j = l / D, k = l - j * D;
    const T* in = bufA + el * SZ_A + l;
    T sg[Q], sb[Q];
#pragma unroll
    for (int qx = 0; qx < Q; ++qx) {
      sg[qx] = in[qx * S_DD];
      if constexpr (DIFF) sb[qx] = in[Q * S_DD + qx * S_DD];
    }
    T* out = bufB + el * SZ_B + j * D + k * D2;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      T r = Ar::zero();
#pragma unroll
      for (int qx = 0; qx < Q; ++qx) {
        if constexpr (DIFF) {
          Ar::madG(r, tab, qx, i, sg[qx]);
          Ar::madB(r, tab, qx, i, sb[qx]);
        } else {
          Ar::madB(r, tab, qx, i, sg[qx]);
        }
      }
      out[i] = r;
    }
  }
  __syncthreads();

  // ---- scatter-add (G^T)
  for (int t = tid; t < nel * D3; t += NT) {
    const int el = t / D3, a = t - el * D3;
    const int32_t g = __ldg(&map[(e0 + el) * D3 + a]);
    Ar::scatter(&y[g], bufB[el * SZ_B + a]);
  }
}

}  // namespace fe
