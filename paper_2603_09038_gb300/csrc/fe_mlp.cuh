// BF16 tensor-core GEMM and elementwise kernels of the learned patch preconditioner.
//
// C[M x N] (FP32) = op(A) op(B) with A, B in BF16 row-major storage and FP32 accumulation on the
// tensor cores (mma.sync.m16n8k16.row.col.f32.bf16.bf16.f32).  op(A) is A [M x K] or, with
// TA, the transpose of A stored [K x M]; op(B) is B [K x N] or, with TB, the transpose of B
// stored [N x K].  Tiles of 64 x 64 per block of 4 warps (32 x 32 per warp), K in steps of 32
// staged through shared memory (padded rows).  Epilogues: plain FP32 store; ReLU with a BF16 copy
// of the activation (forward); multiplication by the ReLU mask of a stored pre-activation
// (backward).  Fragment layouts of m16n8k16 (g = lane / 4, t = lane % 4): A rows g and g + 8,
// columns 2t, 2t + 1 (+ 8); B columns g, rows 2t, 2t + 1 (+ 8); C rows g, g + 8, columns 2t, 2t + 1.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>


namespace fe {
namespace mlp {

constexpr int BM = 64, BN = 64, BK = 32, KPAD = 8, GEMM_THREADS = 128;

enum Epi { EPI_STORE = 0, EPI_RELU_BF16 = 1, EPI_RELU_MASK_BF16 = 2, EPI_ACCUM = 3 };

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4],
                                         const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// EPI_STORE:          C = acc (FP32, ldc)
// EPI_ACCUM:          C += acc
// EPI_RELU_BF16:      C = acc (pre-activation, FP32; skipped if C is null) and Hb = bf16(relu(acc))
// EPI_RELU_MASK_BF16: Hb = bf16(acc * (Z > 0)) with Z the stored pre-activation (ldc)
template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(GEMM_THREADS) k_gemm_bf16(
    int M, int N, int K, const __nv_bfloat16* __restrict__ A, int lda,
    const __nv_bfloat16* __restrict__ B, int ldb, float* __restrict__ C, int ldc,
    __nv_bfloat16* __restrict__ Hb, int ldh) {
  __shared__ __nv_bfloat16 sA[BM][BK + KPAD];  // [m][k]
  __shared__ __nv_bfloat16 sB[BN][BK + KPAD];  // [n][k]
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
  const int wm = (warp / 2) * 32, wn = (warp % 2) * 32;
  const int g = lane / 4, t = lane % 4;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[i][j][c] = 0.0f;
  const __nv_bfloat16 zero = __float2bfloat16(0.0f);
  for (int k0 = 0; k0 < K; k0 += BK) {
    for (int idx = tid; idx < BM * BK; idx += GEMM_THREADS) {
      int m, k;
      if (TA) {  // A stored [K][M]: consecutive threads walk m
        m = idx % BM;
        k = idx / BM;
      } else {
        k = idx % BK;
        m = idx / BK;
      }
      const int gm = m0 + m, gk = k0 + k;
      __nv_bfloat16 v = zero;
      if (gm < M && gk < K) v = TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
      sA[m][k] = v;
    }
    for (int idx = tid; idx < BN * BK; idx += GEMM_THREADS) {
      int n, k;
      if (TB) {  // B stored [N][K]
        k = idx % BK;
        n = idx / BK;
      } else {   // B stored [K][N]
        n = idx % BN;
        k = idx / BN;
      }
      const int gn = n0 + n, gk = k0 + k;
      __nv_bfloat16 v = zero;
      if (gn < N && gk < K) v = TB ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn];
      sB[n][k] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      uint32_t af[2][4], bfr[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm + i * 16 + g;
        af[i][0] = pack2(sA[r][kk + 2 * t], sA[r][kk + 2 * t + 1]);
        af[i][1] = pack2(sA[r + 8][kk + 2 * t], sA[r + 8][kk + 2 * t + 1]);
        af[i][2] = pack2(sA[r][kk + 2 * t + 8], sA[r][kk + 2 * t + 9]);
        af[i][3] = pack2(sA[r + 8][kk + 2 * t + 8], sA[r + 8][kk + 2 * t + 9]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int cn = wn + j * 8 + g;
        bfr[j][0] = pack2(sB[cn][kk + 2 * t], sB[cn][kk + 2 * t + 1]);
        bfr[j][1] = pack2(sB[cn][kk + 2 * t + 8], sB[cn][kk + 2 * t + 9]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma16816(acc[i][j], af[i], bfr[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int row = m0 + wm + i * 16 + g + (c >= 2 ? 8 : 0);
        const int col = n0 + wn + j * 8 + 2 * t + (c & 1);
        if (row >= M || col >= N) continue;
        const float v = acc[i][j][c];
        if (EPI == EPI_STORE) {
          C[(size_t)row * ldc + col] = v;
        } else if (EPI == EPI_ACCUM) {
          C[(size_t)row * ldc + col] += v;
        } else if (EPI == EPI_RELU_BF16) {
          if (C) C[(size_t)row * ldc + col] = v;
          Hb[(size_t)row * ldh + col] = __float2bfloat16(v > 0.0f ? v : 0.0f);
        } else {
          const float z = C[(size_t)row * ldc + col];
          Hb[(size_t)row * ldh + col] = __float2bfloat16(z > 0.0f ? v : 0.0f);
        }
      }
}

template <bool TA, bool TB, int EPI>
inline cudaError_t gemm(int M, int N, int K, const __nv_bfloat16* A, int lda,
                        const __nv_bfloat16* B, int ldb, float* C, int ldc, __nv_bfloat16* Hb,
                        int ldh, cudaStream_t s) {
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
  k_gemm_bf16<TA, TB, EPI><<<grid, GEMM_THREADS, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, Hb, ldh);
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------------------------
// Fused inference of the patch preconditioner: z += sum_e R_e^T F_e s_e f(x_e / s_e),
// x_e = F_e R_e r, s_e = ||x_e||_2, F = the per-dof input/output scaling (0 on the boundary), and
// f(x) = relu(relu(x W1) W2) W3 + x W0.  One warp per tile of 16 elements (rows): the gather
// writes the normalised BF16 rows to the warp's shared staging tile, layer 1 and the skip term
// read their A fragments from it, and every later layer takes its A fragments straight from the
// previous layer's FP32 accumulators (the m16n8 C layout of two adjacent n-tiles is the m16n8k16
// A layout), so no activation leaves the registers.  The weights live in shared memory for the
// whole (persistent) kernel as BF16 images [n][k] (k contiguous, 32-bit words XOR-swizzled by
// n mod 8 so that the 8 x 4 fragment loads of a warp hit 32 distinct banks), made once per weight
// update by k_pack_wimg.  DP = D^3 rounded up to a multiple of 16, W = width (a multiple of 64,
// or 0 for the linear patch map f(x) = x W0).

__host__ __device__ constexpr int fused_dp(int din) { return (din + 15) / 16 * 16; }

__device__ __forceinline__ int swz(int n, int kw, int kwords) {
  return kw ^ (((n & 7) << 2) & (kwords - 1));
}

template <int DP, int W>
struct FusedLayout {
  static constexpr int W1 = 0;                // [W][DP]
  static constexpr int W2 = W1 + W * DP;      // [W][W]
  static constexpr int W3 = W2 + W * W;       // [DP][W]
  static constexpr int W0 = W3 + DP * W;      // [DP][DP]
  static constexpr int WELEMS = W0 + DP * DP; // BF16 elements of the weight image
  static constexpr int WARPS = 8;
  static constexpr int XS = 16 * DP;          // staging tile per warp (BF16 elements)
  static constexpr size_t SMEM = (size_t)(WELEMS + WARPS * XS) * 2 + WARPS * 16 * sizeof(float);
};

// Offsets (in BF16 elements) of the four images for runtime sizes (same as FusedLayout).
__host__ __device__ inline void fused_offsets(int DP, int W, int64_t off[5]) {
  off[0] = 0;
  off[1] = off[0] + (int64_t)W * DP;
  off[2] = off[1] + (int64_t)W * W;
  off[3] = off[2] + (int64_t)DP * W;
  off[4] = off[3] + (int64_t)DP * DP;
}

// One BF16 image element per thread: layer L (0..3 = W1, W2, W3, W0) stored [N][K] swizzled, from
// the FP32 master weights (row-major [k][n] with the true sizes; zero padding beyond them).
__global__ void k_pack_wimg(const float* __restrict__ w32, int din, int width, int DP,
                            __nv_bfloat16* __restrict__ img) {
  int64_t off[5];
  fused_offsets(DP, width, off);
  const int64_t src1 = 0, src2 = (int64_t)din * width, src3 = src2 + (int64_t)width * width,
                src0 = src3 + (int64_t)width * din;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < off[4];
       i += (int64_t)gridDim.x * blockDim.x) {
    int L = 0;
    while (i >= off[L + 1]) ++L;
    const int64_t j = i - off[L];
    int K, nv, kv;  // row length of the image, valid rows (n) and valid columns (k)
    int64_t src;
    if (L == 0) { K = DP; nv = width; kv = din; src = src1; }
    else if (L == 1) { K = width; nv = width; kv = width; src = src2; }
    else if (L == 2) { K = width; nv = din; kv = width; src = src3; }
    else { K = DP; nv = din; kv = din; src = src0; }
    const int n = (int)(j / K), k = (int)(j % K);
    const float v = (n < nv && k < kv) ? w32[src + (int64_t)k * nv + n] : 0.0f;
    const int kw = swz(n, k / 2, K / 2);
    img[off[L] + (int64_t)n * K + 2 * kw + (k & 1)] = __float2bfloat16(v);
  }
}

__device__ __forceinline__ uint32_t pack_relu(float lo, float hi) {
  return pack2(__float2bfloat16(lo > 0.0f ? lo : 0.0f), __float2bfloat16(hi > 0.0f ? hi : 0.0f));
}

// Widths up to 128 with D^3 <= 64 are register-capped for two resident blocks per SM (16 warps
// to hide the gather's memory latency); larger tiles need the full register file of one block;
// the linear map (W = 0) runs three blocks per SM (two for D^3 > 64).
// VT: element type of the r and z vectors (double; float inside the mixed-precision solver).
template <int DP, int W, class VT>
__global__ void __launch_bounds__(256, (W == 0 ? (DP <= 64 ? 3 : 2) : (W <= 128 && DP <= 64 ? 2 : 1))) k_lpc_fused(
    const uint4* __restrict__ wimg, const VT* __restrict__ r, const int32_t* __restrict__ map,
    const float* __restrict__ fsc, int64_t ne, int din, VT* __restrict__ z) {
  using Lay = FusedLayout<DP, W>;
  static_assert(W % 64 == 0 && DP % 16 == 0, "fused MLP tile sizes");
  constexpr int DPW = DP / 2, WW = W > 0 ? W / 2 : 1;  // 32-bit words per image row
  constexpr int WPL = (DPW + 31) / 32;      // staging words per lane in the gather
  constexpr int GR = 8 / WPL;               // rows gathered per step (loads in flight)
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* sw = reinterpret_cast<uint32_t*>(smem);
  {
    uint4* sv = reinterpret_cast<uint4*>(smem);
    for (int i = threadIdx.x; i < Lay::WELEMS / 8; i += blockDim.x) sv[i] = wimg[i];
  }
  __syncthreads();
  const uint32_t* W1s = sw + Lay::W1 / 2;
  const uint32_t* W2s = sw + Lay::W2 / 2;
  const uint32_t* W3s = sw + Lay::W3 / 2;
  const uint32_t* W0s = sw + Lay::W0 / 2;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, g = lane / 4, t = lane % 4;
  uint32_t* xs = sw + Lay::WELEMS / 2 + warp * (Lay::XS / 2);
  float* ssc = reinterpret_cast<float*>(sw + Lay::WELEMS / 2 + Lay::WARPS * (Lay::XS / 2)) + warp * 16;
  const int64_t ntiles = (ne + 15) / 16;
  for (int64_t tile = (int64_t)blockIdx.x * Lay::WARPS + warp; tile < ntiles;
       tile += (int64_t)gridDim.x * Lay::WARPS) {
    // ---- gather: x = F r on the element, normalised, to BF16 (GR rows at a time for ILP).  The
    // FP64 inputs are narrowed to floats (one conversion each; the scaling F is stored in FP32)
    // and the scaling is done in FP32:
    // with FP64 arithmetic here GB300's FP64 pipe (2 DFMA per clock per SM) bound the kernel
    // (81 % busy); narrowing by integer manipulation instead of the conversion instruction was
    // measured slower (more instructions in a latency-bound kernel), for the MLP and for the
    // linear map alike.
#pragma unroll 1
    for (int i0 = 0; i0 < 16; i0 += GR) {
      float xv[GR][WPL][2];
#pragma unroll
      for (int i = 0; i < GR; ++i) {
        const int64_t e = tile * 16 + i0 + i;
#pragma unroll
        for (int w = 0; w < WPL; ++w) {
          const int kw = lane + 32 * w;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int k = 2 * kw + h;
            float v = 0.0f;
            if (kw < DPW && k < din && e < ne) {
              const int32_t idx = map[e * din + k];
              v = fsc[idx] * (float)r[idx];
            }
            xv[i][w][h] = v;
          }
        }
      }
#pragma unroll
      for (int i = 0; i < GR; ++i) {
        // ||x|| from the largest magnitude m: sum (x/m)^2 cannot overflow or underflow
        float mx = 0.0f;
#pragma unroll
        for (int w = 0; w < WPL; ++w) mx = fmaxf(mx, fmaxf(fabsf(xv[i][w][0]), fabsf(xv[i][w][1])));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        const float im = mx > 0.0f ? 1.0f / mx : 0.0f;
        float ss = 0.0f;
#pragma unroll
        for (int w = 0; w < WPL; ++w) {
          const float a0 = xv[i][w][0] * im, a1 = xv[i][w][1] * im;
          ss = fmaf(a0, a0, fmaf(a1, a1, ss));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        const float sn = sqrtf(ss);               // ||x|| / m, in [1, 8 sqrt(2)]
        const float inv = mx > 0.0f ? im / sn : 0.0f;
        const int row = i0 + i;
#pragma unroll
        for (int w = 0; w < WPL; ++w) {
          const int kw = lane + 32 * w;
          if (kw < DPW)
            xs[row * DPW + swz(row, kw, DPW)] = pack2(__float2bfloat16(xv[i][w][0] * inv),
                                                      __float2bfloat16(xv[i][w][1] * inv));
        }
        if (lane == 0) ssc[row] = mx * sn;
      }
    }
    __syncwarp();
    float y[DP / 8][4];
#pragma unroll
    for (int j = 0; j < DP / 8; ++j) y[j][0] = y[j][1] = y[j][2] = y[j][3] = 0.0f;
    if constexpr (W > 0) {  // width 0: the linear patch map x W0 alone
    // ---- layer 1: h1 = relu(x W1), 64 output columns at a time
    uint32_t h1[W / 16][4];
#pragma unroll
    for (int c = 0; c < W / 64; ++c) {
      float acc[8][4];
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
#pragma unroll
      for (int kk = 0; kk < DP / 16; ++kk) {
        const uint32_t a[4] = {xs[g * DPW + swz(g, kk * 8 + t, DPW)],
                               xs[(g + 8) * DPW + swz(g + 8, kk * 8 + t, DPW)],
                               xs[g * DPW + swz(g, kk * 8 + 4 + t, DPW)],
                               xs[(g + 8) * DPW + swz(g + 8, kk * 8 + 4 + t, DPW)]};
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int n = c * 64 + j * 8 + g;
          const uint32_t b[2] = {W1s[n * DPW + swz(n, kk * 8 + t, DPW)],
                                 W1s[n * DPW + swz(n, kk * 8 + 4 + t, DPW)]};
          mma16816(acc[j], a, b);
        }
      }
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        h1[c * 4 + jj][0] = pack_relu(acc[2 * jj][0], acc[2 * jj][1]);
        h1[c * 4 + jj][1] = pack_relu(acc[2 * jj][2], acc[2 * jj][3]);
        h1[c * 4 + jj][2] = pack_relu(acc[2 * jj + 1][0], acc[2 * jj + 1][1]);
        h1[c * 4 + jj][3] = pack_relu(acc[2 * jj + 1][2], acc[2 * jj + 1][3]);
      }
    }
    // ---- layer 2: h2 = relu(h1 W2)
    uint32_t h2[W / 16][4];
#pragma unroll
    for (int c = 0; c < W / 64; ++c) {
      float acc[8][4];
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
#pragma unroll
      for (int kk = 0; kk < W / 16; ++kk) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int n = c * 64 + j * 8 + g;
          const uint32_t b[2] = {W2s[n * WW + swz(n, kk * 8 + t, WW)],
                                 W2s[n * WW + swz(n, kk * 8 + 4 + t, WW)]};
          mma16816(acc[j], h1[kk], b);
        }
      }
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        h2[c * 4 + jj][0] = pack_relu(acc[2 * jj][0], acc[2 * jj][1]);
        h2[c * 4 + jj][1] = pack_relu(acc[2 * jj][2], acc[2 * jj][3]);
        h2[c * 4 + jj][2] = pack_relu(acc[2 * jj + 1][0], acc[2 * jj + 1][1]);
        h2[c * 4 + jj][3] = pack_relu(acc[2 * jj + 1][2], acc[2 * jj + 1][3]);
      }
    }
    // ---- layer 3: y = h2 W3
#pragma unroll
    for (int kk = 0; kk < W / 16; ++kk) {
#pragma unroll
      for (int j = 0; j < DP / 8; ++j) {
        const int n = j * 8 + g;
        const uint32_t b[2] = {W3s[n * WW + swz(n, kk * 8 + t, WW)],
                               W3s[n * WW + swz(n, kk * 8 + 4 + t, WW)]};
        mma16816(y[j], h2[kk], b);
      }
    }
    }  // W > 0
    // ---- the skip term: y += x W0
#pragma unroll
    for (int kk = 0; kk < DP / 16; ++kk) {
      const uint32_t a[4] = {xs[g * DPW + swz(g, kk * 8 + t, DPW)],
                             xs[(g + 8) * DPW + swz(g + 8, kk * 8 + t, DPW)],
                             xs[g * DPW + swz(g, kk * 8 + 4 + t, DPW)],
                             xs[(g + 8) * DPW + swz(g + 8, kk * 8 + 4 + t, DPW)]};
#pragma unroll
      for (int j = 0; j < DP / 8; ++j) {
        const int n = j * 8 + g;
        const uint32_t b[2] = {W0s[n * DPW + swz(n, kk * 8 + t, DPW)],
                               W0s[n * DPW + swz(n, kk * 8 + 4 + t, DPW)]};
        mma16816(y[j], a, b);
      }
    }
    // ---- scatter: z += F s y
    const float s_lo = ssc[g], s_hi = ssc[g + 8];
#pragma unroll
    for (int j = 0; j < DP / 8; ++j) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int row = g + (c >= 2 ? 8 : 0);
        const int col = j * 8 + 2 * t + (c & 1);
        const int64_t e = tile * 16 + row;
        if (col < din && e < ne) {
          const int32_t idx = map[e * din + col];
          const float f = fsc[idx];
          if (f != 0.0f)
            atomicAdd(&z[idx], (VT)(f * (c >= 2 ? s_hi : s_lo) * y[j][c]));
        }
      }
    }
    __syncwarp();  // the staging tile is rewritten by the next tile's gather
  }
}

}  // namespace mlp
}  // namespace fe
