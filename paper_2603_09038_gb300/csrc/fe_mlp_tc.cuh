// Fused inference of the learned patch preconditioner on the 5th-generation tensor cores
// (tcgen05.mma with TMEM accumulators; sm_100-family, built here for sm_103a).
//
// z += sum_e R_e^T F_e s_e f(x_e / s_e), x_e = F_e R_e r, s_e = ||x_e||_2, with
// f(x) = relu(relu(x W1) W2) W3 + x W0 (W = 0: the linear patch map f(x) = x W0) -- the same
// operator as mlp::k_lpc_fused, re-tiled for tcgen05:
//   * a tile of 128 elements (the 128 rows of every layer's M = 128 MMA) is taken by a pipeline
//     of 8 warps; a CTA runs two pipelines on interleaved tiles where their shared memory fits
//     (their own operand tiles, TMEM columns, mbarriers and named barriers), so that one gathers
//     or scatters while the other waits, and they share one copy of the weights;
//   * at width 256 the weights alone nearly fill shared memory: one pipeline of 16 warps keeps
//     the hidden activations in tensor memory instead (ReLU's BF16 output stored by tcgen05.st
//     beside the accumulator, read back by the next layer's MMA as its A operand);
//   * the weights live in shared memory for the whole persistent kernel, copied once by
//     cp.async.bulk behind an mbarrier, as BF16 images in the tensor core's canonical K-major
//     layout without swizzle (8-row x 16-byte core matrices, element (n, k) of an N x K image at
//     ((n/8)(K/8) + k/8) 128 + (n%8) 16 + (k%8) 2 bytes: K-adjacent core matrices 128 bytes
//     apart (the descriptor's leading offset), 8-row groups K/8 x 128 bytes apart (its stride
//     offset));
//   * the gather writes the normalised BF16 rows (the A operand of layer 1 and of the skip term)
//     into the same layout; one thread issues each layer's chain of K = 16 MMAs into a FP32
//     accumulator of 128 TMEM lanes x N columns and commits it to an mbarrier; the epilogue
//     warps read their lane quadrant back with tcgen05.ld, apply ReLU and write the BF16 A
//     operand of the next layer; layer 3 and the skip term accumulate into the same columns;
//   * the result goes through a shared staging tile (in two 64-row passes at width 256, where
//     only X's space is free for it) so that the scatter's dof-map reads and atomic adds are
//     warp-coalesced along each element's dofs.
// Every wait on an mbarrier has an iteration limit: on expiry the kernel raises a device flag,
// all threads leave the tile loop together, and the TMEM is freed before the kernel returns.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fe {
namespace mlptc {

constexpr int kRows = 128;     // rows (elements) per tile: the MMA's M
constexpr int kMaxSmemCta = 232448;  // 227 KB of dynamic shared memory per CTA
constexpr long long kWaitLimit = 1ll << 22;  // mbarrier polls before a wait is given up

__host__ __device__ constexpr int pow2_cols(int n) {
  int c = 32;
  while (c < n) c *= 2;
  return c;
}

// Byte offsets of the shared-memory regions for (DP, W), G tile pipelines per CTA and the place
// of the hidden activations (AT: in tensor memory, as the A operand of the next layer; else in
// shared memory): the weight images once, then per pipeline g its operand tiles (X, and H unless
// AT; the staging tile aliases them after the last MMA), its row scales and its mbarrier.
template <int DP, int W, int G, bool AT>
struct TcLayout {
  static constexpr int W1 = 0;                           // [W][DP]
  static constexpr int W2 = W1 + W * DP * 2;             // [W][W]
  static constexpr int W3 = W2 + W * W * 2;              // [DP][W]
  static constexpr int W0 = W3 + DP * W * 2;             // [DP][DP]
  static constexpr int WBYTES = W0 + DP * DP * 2;        // weight images
  static constexpr int YS = DP + 4;                      // staging row stride (floats)
  static constexpr int YROWS = AT ? kRows / 2 : kRows;   // rows staged per scatter pass
  static constexpr int OPND = kRows * (DP + (AT ? 0 : W)) * 2;
  static constexpr int ACT = OPND > YROWS * YS * 4 ? OPND : YROWS * YS * 4;
  static constexpr int GROUP = ACT + kRows * 4;          // one pipeline's region
  static constexpr int X = WBYTES;                       // + g GROUP: [128][DP] BF16
  static constexpr int H = X + kRows * DP * 2;           // + g GROUP: [128][W] BF16 (not AT)
  static constexpr int SCALE = X + ACT;                  // + g GROUP: float[128]
  static constexpr int BAR = WBYTES + G * GROUP;         // weight mbarrier, one per pipeline
  static constexpr int SLOT = BAR + 8 * (1 + G);         // TMEM base address
  static constexpr int SMEM = SLOT + 16;
  // TMEM columns of one pipeline: the FP32 accumulator (max(W, DP) columns), and with AT the
  // BF16 activations after it (two per 32-bit column)
  static constexpr int ACC = pow2_cols(W > DP ? W : DP);
  static constexpr int ACOL = AT ? ACC : 0;              // first activation column
  static constexpr int NC = pow2_cols(ACC + (AT ? W / 2 : 0));
  static constexpr int NCOLS = G * NC;                   // allocated per CTA
  static_assert(DP % 16 == 0 && W % 16 == 0 && DP >= 16 && DP <= 256 && W <= 256,
                "tcgen05 tile sizes: N and K multiples of 16, N <= 256");
  static_assert(WBYTES % 16 == 0 && GROUP % 16 == 0 && (kRows * DP * 2) % 16 == 0,
                "16-byte aligned regions");
  static_assert(NCOLS <= 512, "tensor memory columns");
  static_assert(!AT || G == 1, "activations in tensor memory take all of it: one pipeline");
};

// How (DP, W) is built: two pipelines of 8 warps with the activations in shared memory where
// they fit (one gathers or scatters while the other waits on its tensor-core chain, sharing the
// weights); else one such pipeline; else (the widest layers, whose weights alone nearly fill
// shared memory) one pipeline of 16 warps keeping the activations in tensor memory.
template <int DP, int W>
struct TcConfig {
  static constexpr bool TWO = TcLayout<DP, W, 2, false>::SMEM <= kMaxSmemCta;
  static constexpr bool ONE = TcLayout<DP, W, 1, false>::SMEM <= kMaxSmemCta;
  static constexpr int G = TWO ? 2 : 1;
  static constexpr bool AT = !TWO && !ONE;
  static constexpr int WPG = AT ? 16 : 8;                // warps per pipeline
  using Lay = TcLayout<DP, W, G, AT>;
  static constexpr bool FITS = Lay::SMEM <= kMaxSmemCta;
  static constexpr int THREADS = G * WPG * 32;
};

// Host: offsets (BF16 elements) of the four images in the packed weight buffer.
__host__ __device__ inline void tc_offsets(int DP, int W, int64_t off[5]) {
  off[0] = 0;
  off[1] = off[0] + (int64_t)W * DP;
  off[2] = off[1] + (int64_t)W * W;
  off[3] = off[2] + (int64_t)DP * W;
  off[4] = off[3] + (int64_t)DP * DP;
}

// Element (n, k) of an N x K BF16 image in the canonical K-major layout (BF16 elements).
__host__ __device__ inline int64_t canon(int n, int k, int K) {
  return ((int64_t)(n >> 3) * (K >> 3) + (k >> 3)) * 64 + (n & 7) * 8 + (k & 7);
}

// One image element per thread: layer L (0..3 = W1, W2, W3, W0) from the FP32 master weights
// (row-major [k][n] with the true sizes; zero padding beyond them), as for k_pack_wimg.
__global__ void k_pack_tc(const float* __restrict__ w32, int din, int width, int DP,
                          __nv_bfloat16* __restrict__ img) {
  int64_t off[5];
  tc_offsets(DP, width, off);
  const int64_t src2 = (int64_t)din * width, src3 = src2 + (int64_t)width * width,
                src0 = src3 + (int64_t)width * din;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < off[4];
       i += (int64_t)gridDim.x * blockDim.x) {
    int L = 0;
    while (i >= off[L + 1]) ++L;
    const int64_t j = i - off[L];
    int K, nv, kv;
    int64_t src;
    if (L == 0) { K = DP; nv = width; kv = din; src = 0; }
    else if (L == 1) { K = width; nv = width; kv = width; src = src2; }
    else if (L == 2) { K = width; nv = din; kv = width; src = src3; }
    else { K = DP; nv = din; kv = din; src = src0; }
    const int n = (int)(j / K), k = (int)(j % K);
    const float v = (n < nv && k < kv) ? w32[src + (int64_t)k * nv + n] : 0.0f;
    img[off[L] + canon(n, k, K)] = __float2bfloat16(v);
  }
}

// ---- PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start address, leading (K-direction) and stride (8-row
// direction) byte offsets, the fixed version bits 46-48 = 0b001, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
         ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A and B (bits 7-9
// and 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               ::"r"(bar) : "memory");
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// generic-proxy writes to shared memory made visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void bar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Bounded wait for the phase with parity `parity` of the mbarrier: 1 if it completed.
__device__ __forceinline__ int bar_wait(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  for (long long it = 0; it < kWaitLimit; ++it) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    if (done) return 1;
  }
  return 0;
}

// The calling thread's share of an expected transaction byte count, and its arrival.
__device__ __forceinline__ void bar_arrive_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

// Bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16), completing
// `bytes` transactions on the mbarrier.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
               ::"r"(slot), "r"(ncols) : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

// NCOL (8, 16 or 32) consecutive FP32 columns of the calling thread's TMEM lane (32x32b shape:
// warp w reads lanes 32 (w % 4) .. 32 (w % 4) + 31, thread t lane 32 (w % 4) + t).  The load and
// its wait are one asm statement, so no use of the registers can be scheduled before the wait.
template <int NCOL>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float* v) {
  uint32_t r[NCOL];
  if constexpr (NCOL == 8) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7])
        : "r"(taddr) : "memory");
  } else if constexpr (NCOL == 16) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr) : "memory");
  } else {
    static_assert(NCOL == 32, "8, 16 or 32 columns");
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr) : "memory");
  }
#pragma unroll
  for (int i = 0; i < NCOL; ++i) v[i] = __uint_as_float(r[i]);
}

// Columns per TMEM load when the NQ warps of a lane quadrant share N columns in interleaved
// chunks: as wide as the share allows, at most 32.
__host__ __device__ constexpr int ld_cols(int N, int NQ) {
  return N / NQ >= 32 ? 32 : (N / NQ >= 16 ? 16 : 8);
}

// Barrier of one pipeline's nt threads (named barrier 1 + g; barrier 0 is __syncthreads), and
// the same with an OR-vote of v over them.
__device__ __forceinline__ void group_sync(int g, int nt) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(nt) : "memory");
}
__device__ __forceinline__ int group_or(int g, int nt, int v) {
  int r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.s32 q, %1, 0;\n\t"
      "bar.red.or.pred p, %2, %3, q;\n\tselp.s32 %0, 1, 0, p;\n\t}"
      : "=r"(r) : "r"(v), "r"(1 + g), "r"(nt) : "memory");
  return r;
}

// 8 consecutive 32-bit columns of the calling thread's TMEM lane, stored (the 32x32b shape of
// tmem_ld), and complete before return.
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&w)[8]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
      ::"r"(taddr), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]),
        "r"(w[7])
      : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// D (+)= A B^T with A[128 x 16] in tensor memory (row i in lane i, two BF16 per 32-bit column,
// the lower half first) and B in shared memory.
__device__ __forceinline__ void mma_bf16_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t b,
                                            uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}"
      ::"r"(tmem_d), "r"(tmem_a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16(lo)) |
         ((uint32_t)__bfloat16_as_ushort(__float2bfloat16(hi)) << 16);
}

// One elected thread issues the K / 16 MMAs of D[128 x N] (+)= A[128 x K] B[N x K]^T, both
// operands canonical K-major images in shared memory (K-adjacent core matrices 128 bytes apart,
// 8-row groups K / 8 x 128 bytes apart; a K = 16 step advances the start by two core matrices).
__device__ __forceinline__ void issue_chain(uint32_t tmem, uint32_t a, uint32_t b, int K, int N,
                                            bool accumulate) {
  const uint32_t id = idesc_bf16(kRows, N), sbo = (uint32_t)(K / 8) * 128u;
  for (int kk = 0; kk < K / 16; ++kk)
    mma_bf16(tmem, sdesc(a + kk * 256u, 128u, sbo), sdesc(b + kk * 256u, 128u, sbo), id,
             (accumulate || kk > 0) ? 1u : 0u);
}

// The same with A in tensor memory from column a (a K = 16 step advances it by 8 columns).
__device__ __forceinline__ void issue_chain_ts(uint32_t tmem, uint32_t a, uint32_t b, int K,
                                               int N, bool accumulate) {
  const uint32_t id = idesc_bf16(kRows, N), sbo = (uint32_t)(K / 8) * 128u;
  for (int kk = 0; kk < K / 16; ++kk)
    mma_bf16_ts(tmem, a + 8u * kk, sdesc(b + kk * 256u, 128u, sbo), id,
                (accumulate || kk > 0) ? 1u : 0u);
}

// Epilogues of a hidden layer: the thread's TMEM lane (its tile row), ReLU, BF16, as the next
// layer's A operand; the NQ warps of a lane quadrant take interleaved chunks of CW columns (part
// = this warp's rank among them), one TMEM load each.  Into the canonical [128][N] image at dst
// in shared memory:
template <int N, int NQ>
__device__ __forceinline__ void relu_to_image(uint32_t t_lane, int row, int part,
                                              unsigned char* dst) {
  constexpr int CW = ld_cols(N, NQ);
#pragma unroll
  for (int c = CW * part; c < N; c += CW * NQ) {
    float v[CW];
    tmem_ld<CW>(t_lane + (uint32_t)c, v);
#pragma unroll
    for (int j = 0; j < CW; j += 8) {
      uint4 pk;
      pk.x = pack_bf16(fmaxf(v[j + 0], 0.f), fmaxf(v[j + 1], 0.f));
      pk.y = pack_bf16(fmaxf(v[j + 2], 0.f), fmaxf(v[j + 3], 0.f));
      pk.z = pack_bf16(fmaxf(v[j + 4], 0.f), fmaxf(v[j + 5], 0.f));
      pk.w = pack_bf16(fmaxf(v[j + 6], 0.f), fmaxf(v[j + 7], 0.f));
      *reinterpret_cast<uint4*>(dst + canon(row, c + j, N) * 2) = pk;
    }
  }
}
// or into tensor memory from column acol of the same lane (16 values per 8 columns).
template <int N, int NQ>
__device__ __forceinline__ void relu_to_tmem(uint32_t t_lane, int part, uint32_t acol) {
  constexpr int CW = ld_cols(N, NQ) < 16 ? 16 : ld_cols(N, NQ);
  static_assert(N % (CW * NQ) == 0, "whole chunks");
#pragma unroll
  for (int c = CW * part; c < N; c += CW * NQ) {
    float v[CW];
    tmem_ld<CW>(t_lane + (uint32_t)c, v);
#pragma unroll
    for (int j = 0; j < CW; j += 16) {
      uint32_t w[8];
#pragma unroll
      for (int i = 0; i < 8; ++i)
        w[i] = pack_bf16(fmaxf(v[j + 2 * i], 0.f), fmaxf(v[j + 2 * i + 1], 0.f));
      tmem_st8(t_lane + acol + (uint32_t)((c + j) / 2), w);
    }
  }
}

// VT: element type of r and z (double; float inside the mixed-precision solver).  fail: device
// flag raised when a wait on the tensor core or on the weight copy is given up.  G pipelines of
// WPG warps per CTA; AT: hidden activations in tensor memory (TcConfig).
template <int DP, int W, class VT, int G, bool AT, int WPG>
__global__ void __launch_bounds__(G * WPG * 32, 1) k_lpc_tc(
    const __nv_bfloat16* __restrict__ wimg, const VT* __restrict__ r,
    const int32_t* __restrict__ map, const float* __restrict__ fsc, int64_t ne, int din,
    VT* __restrict__ z, int* __restrict__ fail) {
  using Lay = TcLayout<DP, W, G, AT>;
  constexpr int GT = WPG * 32;             // threads of one pipeline
  constexpr int NQ = WPG / 4;              // its warps per TMEM lane quadrant
  constexpr int RPW = kRows / WPG;         // tile rows per warp in the gather
  constexpr int SPW = Lay::YROWS / WPG;    // staged rows per warp in one scatter pass
  static_assert(WPG % 4 == 0 && RPW >= 4 && SPW >= 4, "pipeline shape");
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // pipeline g: warps WPG g .. WPG g + WPG - 1, its own operand tiles, scales, mbarrier, TMEM
  const int g = warp / WPG, gtid = tid - g * GT, gwarp = warp - g * WPG;
  const uint32_t sb = smem_u32(smem);
  const int gb = g * Lay::GROUP;
  const uint32_t bar_w = sb + Lay::BAR, bar_m = sb + Lay::BAR + 8 * (1 + g);
  uint32_t* slot = reinterpret_cast<uint32_t*>(smem + Lay::SLOT);
  float* sscale = reinterpret_cast<float*>(smem + Lay::SCALE + gb);
  unsigned char* sX = smem + Lay::X + gb;
  unsigned char* sH = smem + Lay::H + gb;
  float* sY = reinterpret_cast<float*>(sX);  // after the last MMA of a tile

  // ---- barriers, TMEM, the weight images (one bulk copy stream behind an mbarrier)
  if (tid == 0) {
    bar_init(bar_w, 1);
    for (int k = 0; k < G; ++k) bar_init(sb + Lay::BAR + 8 * (1 + k), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(smem_u32(slot), Lay::NCOLS);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *slot, tmem_g = tmem + (uint32_t)(g * Lay::NC);
  if (tid == 0) {
    bar_arrive_expect(bar_w, (uint32_t)Lay::WBYTES);
    const unsigned char* src = reinterpret_cast<const unsigned char*>(wimg);
    for (int off = 0; off < Lay::WBYTES; off += 16384) {
      const int n = (Lay::WBYTES - off) < 16384 ? (Lay::WBYTES - off) : 16384;
      bulk_g2s(sb + (uint32_t)off, src + off, (uint32_t)n, bar_w);
    }
  }
  int bad = __syncthreads_or(!bar_wait(bar_w, 0));

  const int q = warp & 3, part = gwarp >> 2;
  const int erow = 32 * q + lane;  // this thread's TMEM lane = tile row in the epilogues
  const uint32_t t_lane = tmem_g + ((uint32_t)(32 * q) << 16);
  uint32_t phase = 0;
  const int64_t ntiles = (ne + kRows - 1) / kRows;
  constexpr int NPAIR = DP / 2, PPL = (NPAIR + 31) / 32;  // BF16 pairs per row, per lane
  constexpr int RG0 = PPL > 1 ? 4 : 8;
  constexpr int RG = RG0 < RPW ? RG0 : RPW;               // rows per gather group
  constexpr int RS = RG0 < SPW ? RG0 : SPW;               // rows per scatter group
  for (int64_t tile = (int64_t)blockIdx.x * G + g; tile < ntiles && !bad;
       tile += (int64_t)gridDim.x * G) {
    // ---- gather: x = F r on each element, normalised by its norm, BF16 into the X image;
    //      warp w takes rows RPW w .. RPW w + RPW - 1, RG at a time: every dof-map entry of the
    //      group is loaded first, then the values, so that all of them are in flight together
#pragma unroll 1
    for (int r0 = RPW * gwarp; r0 < RPW * gwarp + RPW; r0 += RG) {
      int32_t gi[RG][PPL][2];
#pragma unroll
      for (int i = 0; i < RG; ++i) {
        const int64_t e = tile * kRows + r0 + i;
#pragma unroll
        for (int w = 0; w < PPL; ++w)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int k = 2 * (lane + 32 * w) + h;
            gi[i][w][h] = (k < din && e < ne) ? __ldg(&map[e * din + k]) : -1;
          }
      }
      float xv[RG][PPL][2];
#pragma unroll
      for (int i = 0; i < RG; ++i)
#pragma unroll
        for (int w = 0; w < PPL; ++w)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int32_t idx = gi[i][w][h];
            xv[i][w][h] = idx >= 0 ? __ldg(&fsc[idx]) * (float)__ldg(&r[idx]) : 0.0f;
          }
#pragma unroll
      for (int i = 0; i < RG; ++i) {
        float mx = 0.0f;
#pragma unroll
        for (int w = 0; w < PPL; ++w) mx = fmaxf(mx, fmaxf(fabsf(xv[i][w][0]), fabsf(xv[i][w][1])));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        const float im = mx > 0.0f ? 1.0f / mx : 0.0f;
        float ss = 0.0f;
#pragma unroll
        for (int w = 0; w < PPL; ++w) {
          const float a0 = xv[i][w][0] * im, a1 = xv[i][w][1] * im;
          ss = fmaf(a0, a0, fmaf(a1, a1, ss));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        const float sn = sqrtf(ss);  // ||x|| / max |x|
        const float inv = mx > 0.0f ? im / sn : 0.0f;
        const int row = r0 + i;
#pragma unroll
        for (int w = 0; w < PPL; ++w) {
          const int kp = lane + 32 * w;
          if (kp < NPAIR)
            *reinterpret_cast<uint32_t*>(sX + canon(row, 2 * kp, DP) * 2) =
                pack_bf16(xv[i][w][0] * inv, xv[i][w][1] * inv);
        }
        if (lane == 0) sscale[row] = mx * sn;
      }
    }
    fence_proxy_async();
    group_sync(g, GT);

    // ---- the layers: one thread issues, everybody waits on the commit, the epilogue warps
    //      read their lane quadrant back
    if constexpr (W > 0) {
#pragma unroll 1
      for (int layer = 0; layer < 2 && !bad; ++layer) {
        if (gtid == 0) {
          fence_after();
          if (layer == 0)
            issue_chain(tmem_g, sb + Lay::X + gb, sb + Lay::W1, DP, W, false);
          else if constexpr (AT)
            issue_chain_ts(tmem_g, tmem_g + Lay::ACOL, sb + Lay::W2, W, W, false);
          else
            issue_chain(tmem_g, sb + Lay::H + gb, sb + Lay::W2, W, W, false);
          mma_commit(bar_m);
        }
        bad = group_or(g, GT, !bar_wait(bar_m, phase));
        phase ^= 1u;
        if (bad) break;
        fence_after();
        if constexpr (AT) {
          relu_to_tmem<W, NQ>(t_lane, part, (uint32_t)Lay::ACOL);
          fence_before();
        } else {
          relu_to_image<W, NQ>(t_lane, erow, part, sH);
          fence_before();
          fence_proxy_async();
        }
        group_sync(g, GT);
      }
      if (bad) break;
    }
    if (gtid == 0) {
      fence_after();
      issue_chain(tmem_g, sb + Lay::X + gb, sb + Lay::W0, DP, DP, false);  // skip term x W0
      if constexpr (W > 0) {
        if constexpr (AT)
          issue_chain_ts(tmem_g, tmem_g + Lay::ACOL, sb + Lay::W3, W, DP, true);
        else
          issue_chain(tmem_g, sb + Lay::H + gb, sb + Lay::W3, W, DP, true);
      }
      mma_commit(bar_m);
    }
    bad = group_or(g, GT, !bar_wait(bar_m, phase));
    phase ^= 1u;
    if (bad) break;
    fence_after();

    // ---- staging and scatter, Lay::YROWS rows per pass: z += F s y, warp w staged rows
    //      SPW w .. SPW w + SPW - 1, lanes along the element's dofs, RS rows at a time with their
    //      dof-map and scaling loads issued before the adds
#pragma unroll 1
    for (int ph = 0; ph < kRows / Lay::YROWS; ++ph) {
      if (erow / Lay::YROWS == ph) {  // warp-uniform: the quadrant's rows are in this pass
        float* yrow = sY + (erow - ph * Lay::YROWS) * Lay::YS;
        constexpr int CW = ld_cols(DP, NQ);
#pragma unroll
        for (int c = CW * part; c < DP; c += CW * NQ) {
          float v[CW];
          tmem_ld<CW>(t_lane + (uint32_t)c, v);
#pragma unroll
          for (int j = 0; j < CW; j += 4)
            *reinterpret_cast<float4*>(yrow + c + j) = make_float4(v[j], v[j + 1], v[j + 2],
                                                                   v[j + 3]);
        }
      }
      fence_before();
      group_sync(g, GT);
#pragma unroll 1
      for (int s0 = SPW * gwarp; s0 < SPW * gwarp + SPW; s0 += RS) {
        int32_t gi[RS][PPL][2];
#pragma unroll
        for (int i = 0; i < RS; ++i) {
          const int64_t e = tile * kRows + ph * Lay::YROWS + s0 + i;
#pragma unroll
          for (int w = 0; w < PPL; ++w)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int k = 2 * (lane + 32 * w) + h;
              gi[i][w][h] = (k < din && e < ne) ? __ldg(&map[e * din + k]) : -1;
            }
        }
        float fv[RS][PPL][2];
#pragma unroll
        for (int i = 0; i < RS; ++i)
#pragma unroll
          for (int w = 0; w < PPL; ++w)
#pragma unroll
            for (int h = 0; h < 2; ++h)
              fv[i][w][h] = gi[i][w][h] >= 0 ? __ldg(&fsc[gi[i][w][h]]) : 0.0f;
#pragma unroll
        for (int i = 0; i < RS; ++i) {
          const float sc = sscale[ph * Lay::YROWS + s0 + i];
#pragma unroll
          for (int w = 0; w < PPL; ++w)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int k = 2 * (lane + 32 * w) + h;
              if (fv[i][w][h] != 0.0f)
                atomicAdd(&z[gi[i][w][h]], (VT)(fv[i][w][h] * sc * sY[(s0 + i) * Lay::YS + k]));
            }
        }
      }
      group_sync(g, GT);  // the next pass (or tile's gather) rewrites the staging (and X)
    }
  }

  // ---- teardown: a given-up wait is reported, in-flight MMAs get one more bounded wait, and
  //      the TMEM is always freed
  if (bad) {
    if (gtid == 0) atomicExch(fail, 1);
    bar_wait(bar_m, phase);
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    tmem_dealloc(tmem, Lay::NCOLS);
  }
}

}  // namespace mlptc
}  // namespace fe
