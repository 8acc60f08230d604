// FP64 tensor-core variant of the fused apply: every 1D contraction on mma.sync.m8n8k4.f64.
//
// Section III-B of the paper moves the small contractions of the PA kernel from FP64 FMAs to the
// FP64 tensor-core instruction (DMMA) and maps each GEMM's m/n/k onto its own indices
// (Section III-C).  Here each phase of the fused kernel is one GEMM per table,
//     out[m][n] = sum_k T[m][k] in[k][n],
// with m the output 1D index (Q for forward, D for transposed contractions), k the summed index,
// and n the "line" -- every (element, two other indices) position of the phase -- dealt out to
// the warps in tiles of 8.  The 1D tables are the A operands: their fragments are built once per
// warp in registers (zero-padded to 8 x 4 tiles); the B operands come from shared memory in the
// same summed-index-slowest layout the FMA kernel uses; the C fragments are written straight to
// the next phase's layout.  The pointwise D is applied between the forward and transposed z
// GEMMs through a third shared-memory buffer.  Fragment layout of m8n8k4 (Tables III-V):
// lane T holds A[T/4][T%4], B[T%4][T/4] and C[T/4][2(T%4)], C[T/4][2(T%4)+1].
//
// On GB300 the DMMA path runs at ~1.06 TFLOP/s against ~1.2 TFLOP/s for DFMA, and the padding of
// Q, D <= 10 to 8 x 4 tiles wastes half of it or more, so this variant exists to measure the
// paper's technique on this chip, not as the fast path.
#include <mutex>

#include "fe_apply_kernel.cuh"
#include "fe_internal.h"

namespace fe {
namespace {

constexpr int kDmmaThreads = 128;

__device__ __forceinline__ void dmma884(double& c0, double& c1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
               : "+d"(c0), "+d"(c1)
               : "d"(a), "d"(b));
}

constexpr int cdiv(int a, int b) { return (a + b - 1) / b; }

template <int D, int Q, bool DIFF>
struct DmmaLayout {
  using L = ApplyLayout<D, Q, DIFF>;
  static constexpr int SZ_A = L::SZ_A, SZ_B = L::SZ_B;
  static constexpr int SZ_C = L::NC_Q * Q * L::S_QQ;  // g / v at quadrature points [c][qz][line]
  static constexpr int PER_ELEM = SZ_A + SZ_B + SZ_C;
};

// A fragments of a Q x D table used forward (m = q, k = d) or transposed (m = d, k = q).
template <int D, int Q, bool TRANSPOSED>
struct Frag {
  static constexpr int M = TRANSPOSED ? D : Q, K = TRANSPOSED ? Q : D;
  static constexpr int MT = cdiv(M, 8), KT = cdiv(K, 4);
  double a[MT][KT];
  __device__ __forceinline__ void load(const double* tab, int lane) {
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int kt = 0; kt < KT; ++kt) {
        const int m = mt * 8 + lane / 4, k = kt * 4 + lane % 4;
        const int q = TRANSPOSED ? k : m, d = TRANSPOSED ? m : k;
        a[mt][kt] = (m < M && k < K) ? tab[q * D + d] : 0.0;
      }
  }
};

// One warp-level pass over the n-tiles of a phase: for every tile of 8 lines the B operands of
// all k-steps are loaded once (ldB(k, n); zero outside k < K, n < N) and handed to `body`, which
// issues the DMMAs of every table that uses them and stores the C fragments.  The loop bounds
// depend on the warp index only, so every mma.sync is executed by the whole warp.
template <int KT, class LdB, class Body>
__device__ __forceinline__ void for_tiles(int N, int K, int warp, int nwarps, int lane, LdB ldB,
                                          Body body) {
  const int ntiles = (N + 7) / 8;
  for (int nt = warp; nt < ntiles; nt += nwarps) {
    const int nb = nt * 8 + lane / 4;
    double b[KT];
#pragma unroll
    for (int kt = 0; kt < KT; ++kt) {
      const int k = kt * 4 + lane % 4;
      b[kt] = (k < K && nb < N) ? ldB(k, nb) : 0.0;
    }
    body(b, nt * 8 + 2 * (lane % 4));
  }
}

template <int MT, int KT>
__device__ __forceinline__ void mma_tile(const double (&a)[MT][KT], const double* b, int mt,
                                         double& c0, double& c1) {
#pragma unroll
  for (int kt = 0; kt < KT; ++kt) dmma884(c0, c1, a[mt][kt], b[kt]);
}

template <int D, int Q, int NE, bool DIFF>
__global__ void __launch_bounds__(kDmmaThreads) k_pa_apply_dmma(const int32_t* __restrict__ map,
                                                                const double* __restrict__ qd,
                                                                const double* __restrict__ x,
                                                                double* __restrict__ y, int64_t ne,
                                                                const int* __restrict__ skip,
                                                                const __grid_constant__ TabF64<D, Q> tab) {
  using L = ApplyLayout<D, Q, DIFF>;
  using DL = DmmaLayout<D, Q, DIFF>;
  constexpr int D2 = L::D2, D3 = L::D3, Q2 = L::Q2, QD = L::QD;
  constexpr int S_DD = L::S_DD, S_QD = L::S_QD, S_QQ = L::S_QQ;
  constexpr int SZ_A = DL::SZ_A, SZ_B = DL::SZ_B, SZ_C = DL::SZ_C;
  constexpr int NQD = DIFF ? 6 : 1;
  constexpr int NW = kDmmaThreads / 32;
  using FF = Frag<D, Q, false>;
  using FT = Frag<D, Q, true>;

  if (skip != nullptr && *skip != 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* bufA = reinterpret_cast<double*>(smem_raw);
  double* bufB = bufA + NE * SZ_A;
  double* bufC = bufB + NE * SZ_B;
  const int64_t e0 = (int64_t)blockIdx.x * NE;
  const int nel = (int)((ne - e0) < NE ? (ne - e0) : NE);
  const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;

  FF fB, fG;
  FT tB, tG;
  fB.load(tab.B, lane);
  tB.load(tab.B, lane);
  if constexpr (DIFF) {
    fG.load(tab.G, lane);
    tG.load(tab.G, lane);
  }

  // ---- gather: E0[i][j*D + k]
  for (int t = tid; t < nel * D3; t += kDmmaThreads) {
    const int el = t / D3, a = t - el * D3;
    const int i = a % D, j = (a / D) % D, k = a / D2;
    bufA[el * SZ_A + i * S_DD + j * D + k] = __ldg(&x[__ldg(&map[(e0 + el) * D3 + a])]);
  }
  __syncthreads();

  // ---- x phase: m = qx, k = i, n = (el, j*D + k)
  {
    const int N = nel * D2;
    auto ld = [&](int k, int n) { const int el = n / D2; return bufA[el * SZ_A + k * S_DD + (n - el * D2)]; };
    auto st = [&](int m, int n, double v, int c) {
      if (m >= Q || n >= N) return;
      const int el = n / D2, l = n - el * D2, j = l / D, kk = l - j * D;
      bufB[el * SZ_B + c * D * S_QD + j * S_QD + kk * Q + m] = v;
    };
    for_tiles<FF::KT>(N, D, warp, NW, lane, ld, [&](const double* b, int nc) {
#pragma unroll
      for (int mt = 0; mt < FF::MT; ++mt) {
        const int m = mt * 8 + lane / 4;
        double c0 = 0, c1 = 0;
        mma_tile(fB.a, b, mt, c0, c1);
        st(m, nc, c0, 0);
        st(m, nc + 1, c1, 0);
        if constexpr (DIFF) {
          double g0 = 0, g1 = 0;
          mma_tile(fG.a, b, mt, g0, g1);
          st(m, nc, g0, 1);
          st(m, nc + 1, g1, 1);
        }
      }
    });
  }
  __syncthreads();

  // ---- y phase: m = qy, k = j, n = (el, k*Q + qx); c0 = B (G x), c1 = G (B x), c2 = B (B x)
  {
    const int N = nel * QD;
    auto st = [&](int m, int n, double v, int c) {
      if (m >= Q || n >= N) return;
      const int el = n / QD, l = n - el * QD, k = l / Q, qx = l - k * Q;
      bufA[el * SZ_A + c * D * S_QQ + k * S_QQ + m * Q + qx] = v;
    };
    auto ldb = [&](int k, int n) { const int el = n / QD; return bufB[el * SZ_B + k * S_QD + (n - el * QD)]; };
    for_tiles<FF::KT>(N, D, warp, NW, lane, ldb, [&](const double* b, int nc) {
#pragma unroll
      for (int mt = 0; mt < FF::MT; ++mt) {
        const int m = mt * 8 + lane / 4;
        double c0 = 0, c1 = 0;
        if constexpr (DIFF) {
          mma_tile(fG.a, b, mt, c0, c1);
          st(m, nc, c0, 1);
          st(m, nc + 1, c1, 1);
          c0 = c1 = 0;
          mma_tile(fB.a, b, mt, c0, c1);
          st(m, nc, c0, 2);
          st(m, nc + 1, c1, 2);
        } else {
          mma_tile(fB.a, b, mt, c0, c1);
          st(m, nc, c0, 0);
          st(m, nc + 1, c1, 0);
        }
      }
    });
    if constexpr (DIFF) {
      auto ldg = [&](int k, int n) {
        const int el = n / QD;
        return bufB[el * SZ_B + D * S_QD + k * S_QD + (n - el * QD)];
      };
      for_tiles<FF::KT>(N, D, warp, NW, lane, ldg, [&](const double* b, int nc) {
#pragma unroll
        for (int mt = 0; mt < FF::MT; ++mt) {
          const int m = mt * 8 + lane / 4;
          double c0 = 0, c1 = 0;
          mma_tile(fB.a, b, mt, c0, c1);
          st(m, nc, c0, 0);
          st(m, nc + 1, c1, 0);
        }
      });
    }
  }
  __syncthreads();

  // ---- z forward: m = qz, k = k, n = (el, qy*Q + qx) -> bufC[c][qz][line]
  constexpr int NCQ = DIFF ? 3 : 1;
  {
    const int N = nel * Q2;
#pragma unroll
    for (int c = 0; c < NCQ; ++c) {
      auto ld = [&](int k, int n) {
        const int el = n / Q2;
        return bufA[el * SZ_A + c * D * S_QQ + k * S_QQ + (n - el * Q2)];
      };
      for_tiles<FF::KT>(N, D, warp, NW, lane, ld, [&](const double* b, int nc) {
#pragma unroll
        for (int mt = 0; mt < FF::MT; ++mt) {
          const int m = mt * 8 + lane / 4;
          double c0 = 0, c1 = 0;
          if (DIFF && c == 2)
            mma_tile(fG.a, b, mt, c0, c1);
          else
            mma_tile(fB.a, b, mt, c0, c1);
          if (m < Q) {
            if (nc < N) { const int el = nc / Q2; bufC[el * SZ_C + c * Q * S_QQ + m * S_QQ + (nc - el * Q2)] = c0; }
            if (nc + 1 < N) { const int el = (nc + 1) / Q2; bufC[el * SZ_C + c * Q * S_QQ + m * S_QQ + (nc + 1 - el * Q2)] = c1; }
          }
        }
      });
    }
  }
  __syncthreads();

  // ---- pointwise D at every quadrature point (FP64 FMA), in place in bufC
  for (int t = tid; t < nel * Q * Q2; t += kDmmaThreads) {
    const int el = t / (Q * Q2), r = t - el * Q * Q2, qz = r / Q2, l = r - qz * Q2;
    const double* qq = qd + (e0 + el) * (int64_t)(NQD * Q * Q2) + (int64_t)qz * NQD * Q2 + l;
    double* g = bufC + el * SZ_C + qz * S_QQ + l;
    if constexpr (DIFF) {
      const double g0 = g[0], g1 = g[Q * S_QQ], g2 = g[2 * Q * S_QQ];
      const double dxx = __ldcs(qq), dxy = __ldcs(qq + Q2), dxz = __ldcs(qq + 2 * Q2);
      const double dyy = __ldcs(qq + 3 * Q2), dyz = __ldcs(qq + 4 * Q2), dzz = __ldcs(qq + 5 * Q2);
      g[0] = fma(dxz, g2, fma(dxy, g1, dxx * g0));
      g[Q * S_QQ] = fma(dyz, g2, fma(dyy, g1, dxy * g0));
      g[2 * Q * S_QQ] = fma(dzz, g2, fma(dyz, g1, dxz * g0));
    } else {
      g[0] = __ldcs(qq) * g[0];
    }
  }
  __syncthreads();

  // ---- z transposed: m = k, k = qz, n = (el, qy*Q + qx) -> S4c[qy][k*Q + qx] in bufB
  {
    const int N = nel * Q2;
#pragma unroll
    for (int c = 0; c < NCQ; ++c) {
      auto ld = [&](int k, int n) {
        const int el = n / Q2;
        return bufC[el * SZ_C + c * Q * S_QQ + k * S_QQ + (n - el * Q2)];
      };
      for_tiles<FT::KT>(N, Q, warp, NW, lane, ld, [&](const double* b, int nc) {
#pragma unroll
        for (int mt = 0; mt < FT::MT; ++mt) {
          const int m = mt * 8 + lane / 4;
          double c0 = 0, c1 = 0;
          if (DIFF && c == 2)
            mma_tile(tG.a, b, mt, c0, c1);
          else
            mma_tile(tB.a, b, mt, c0, c1);
          if (m < D) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int n = nc + h;
              if (n < N) {
                const int el = n / Q2, l = n - el * Q2, qy = l / Q, qx = l - qy * Q;
                bufB[el * SZ_B + c * Q * S_QD + qy * S_QD + m * Q + qx] = h ? c1 : c0;
              }
            }
          }
        }
      });
    }
  }
  __syncthreads();

  // ---- y^T: m = j, k = qy, n = (el, k*Q + qx) -> S5c[qx][j*D + k]; c0 = B^T s0, c1 = G^T s1 + B^T s2
  {
    const int N = nel * QD;
    auto ldc = [&](int c) {
      return [=](int k, int n) {
        const int el = n / QD;
        return bufB[el * SZ_B + c * Q * S_QD + k * S_QD + (n - el * QD)];
      };
    };
    auto st = [&](int m, int n, double v, int c) {
      if (m >= D || n >= N) return;
      const int el = n / QD, l = n - el * QD, k = l / Q, qx = l - k * Q;
      bufA[el * SZ_A + c * Q * S_DD + qx * S_DD + m * D + k] = v;
    };
    if constexpr (DIFF) {
      // c1 accumulates two GEMMs: G^T s1 first, B^T s2 second, through the same C fragments
      const int ntiles = (N + 7) / 8;
      for (int nt = warp; nt < ntiles; nt += NW) {
        const int nb = nt * 8 + lane / 4, nc = nt * 8 + 2 * (lane % 4);
        double b0[FT::KT], b1[FT::KT], b2[FT::KT];
#pragma unroll
        for (int kt = 0; kt < FT::KT; ++kt) {
          const int k = kt * 4 + lane % 4;
          const bool ok = (k < Q && nb < N);
          b0[kt] = ok ? ldc(0)(k, nb) : 0.0;
          b1[kt] = ok ? ldc(1)(k, nb) : 0.0;
          b2[kt] = ok ? ldc(2)(k, nb) : 0.0;
        }
#pragma unroll
        for (int mt = 0; mt < FT::MT; ++mt) {
          const int m = mt * 8 + lane / 4;
          double c0 = 0, c1 = 0, d0 = 0, d1 = 0;
          mma_tile(tB.a, b0, mt, c0, c1);
          mma_tile(tG.a, b1, mt, d0, d1);
          mma_tile(tB.a, b2, mt, d0, d1);
          st(m, nc, c0, 0);
          st(m, nc + 1, c1, 0);
          st(m, nc, d0, 1);
          st(m, nc + 1, d1, 1);
        }
      }
    } else {
      for_tiles<FT::KT>(N, Q, warp, NW, lane, ldc(0), [&](const double* b, int nc) {
#pragma unroll
        for (int mt = 0; mt < FT::MT; ++mt) {
          const int m = mt * 8 + lane / 4;
          double c0 = 0, c1 = 0;
          mma_tile(tB.a, b, mt, c0, c1);
          st(m, nc, c0, 0);
          st(m, nc + 1, c1, 0);
        }
      });
    }
  }
  __syncthreads();

  // ---- x^T: m = i, k = qx, n = (el, j*D + k) -> Ye[i + D j + D^2 k]; r = G^T sg + B^T sb
  {
    const int N = nel * D2;
    const int ntiles = (N + 7) / 8;
    for (int nt = warp; nt < ntiles; nt += NW) {
      const int nb = nt * 8 + lane / 4, nc = nt * 8 + 2 * (lane % 4);
      double bg[FT::KT], bb[FT::KT];
#pragma unroll
      for (int kt = 0; kt < FT::KT; ++kt) {
        const int k = kt * 4 + lane % 4;
        const bool ok = (k < Q && nb < N);
        const int el = nb / D2;
        const int base = el * SZ_A + k * S_DD + (nb - el * D2);
        bg[kt] = ok ? bufA[base] : 0.0;
        bb[kt] = (ok && DIFF) ? bufA[base + Q * S_DD] : 0.0;
      }
#pragma unroll
      for (int mt = 0; mt < FT::MT; ++mt) {
        const int m = mt * 8 + lane / 4;
        double c0 = 0, c1 = 0;
        if constexpr (DIFF) {
          mma_tile(tG.a, bg, mt, c0, c1);
          mma_tile(tB.a, bb, mt, c0, c1);
        } else {
          mma_tile(tB.a, bg, mt, c0, c1);
        }
        if (m < D) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int n = nc + h;
            if (n < N) {
              const int el = n / D2, l = n - el * D2, j = l / D, kk = l - j * D;
              bufB[el * SZ_B + j * D + kk * D2 + m] = h ? c1 : c0;
            }
          }
        }
      }
    }
  }
  __syncthreads();

  // ---- scatter-add
  for (int t = tid; t < nel * D3; t += kDmmaThreads) {
    const int el = t / D3, a = t - el * D3;
    atomicAdd(&y[__ldg(&map[(e0 + el) * D3 + a])], bufB[el * SZ_B + a]);
  }
}

template <int D, int Q, bool DIFF>
int run_dmma(const ApplyArgs& a, cudaStream_t s) {
  constexpr int bytes = DmmaLayout<D, Q, DIFF>::PER_ELEM * 8;
  constexpr int ne_fit = (96 * 1024) / bytes;
  constexpr int NE = ne_fit >= 16 ? 16 : (ne_fit >= 8 ? 8 : (ne_fit >= 4 ? 4 : (ne_fit >= 2 ? 2 : 1)));
  const size_t smem = (size_t)NE * bytes;
  auto kern = k_pa_apply_dmma<D, Q, NE, DIFF>;
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [&] {
    attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (attr_err != cudaSuccess) return cuda_error(attr_err, "cudaFuncSetAttribute(dmma)");
  TabF64<D, Q> tab;
  for (int i = 0; i < Q * D; ++i) {
    tab.B[i] = a.basis->B[i];
    tab.G[i] = a.basis->G[i];
  }
  const int64_t nblk = (a.ne + NE - 1) / NE;
  if (a.blocks) *a.blocks = nblk;
  if (nblk == 0 || a.query_only) return FE_OK;
  kern<<<(unsigned int)nblk, kDmmaThreads, smem, s>>>(a.map, a.qd, a.x, a.y, a.ne, a.skip, tab);
  return cuda_error(cudaGetLastError(), "dmma apply kernel launch");
}

}  // namespace

int launch_apply_dmma(int op, const ApplyArgs& a, cudaStream_t s) {
  const bool diff = (op == FE_DIFFUSION);
  if (a.Q != a.p + 2) return set_error(FE_ERR_UNSUPPORTED, "only q1d = order + 2 is built");
#define FE_DCASE(P)                                                      \
  case P:                                                                \
    return diff ? run_dmma<P + 1, P + 2, true>(a, s) : run_dmma<P + 1, P + 2, false>(a, s);
  switch (a.p) {
    FE_DCASE(1)
    FE_DCASE(2)
    FE_DCASE(3)
    FE_DCASE(4)
    FE_DCASE(5)
    FE_DCASE(6)
    FE_DCASE(7)
    FE_DCASE(8)
    default:
      return set_error(FE_ERR_UNSUPPORTED, "order out of range 1..8");
  }
#undef FE_DCASE
}

}  // namespace fe
