// Jacobi-preconditioned conjugate gradients with a device-resident state.
//
// The paper has no solver for this operator (it time-steps a wave equation); fe_pcg is the
// standard preconditioned CG (Hestenes-Stiefel) around the fused apply, with the Dirichlet
// boundary handled by the constrained operator A_bc = (1-m) A (1-m) + m.  Started from zero with
// the boundary entries of b ignored, every iterate, residual and search direction stays zero on
// the boundary, so A_bc p reduces to (1-m) A p.
//
// GB300 layout of one iteration (no host round trip): zero q | fused apply q = A p | p.q
// partials | control (alpha) | x, r, z update + r.z, r.r partials | control (beta, stop test) |
// p update.  Scalars and the stop flag live in device memory; every kernel returns at once when
// the flag is set, so the host queues iterations in batches and reads the flag once per batch.
// Inner products are deterministic: a fixed grid of kReduceBlocks blocks, fixed in-block trees,
// and the partials summed in block order by a single thread.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <mutex>
#include <string>

#include "fe_internal.h"

namespace {

using namespace fe;

constexpr int kReduceBlocks = 1024;
constexpr int kReduceThreads = 256;
constexpr int kBatch = 8;  // iterations queued between two host reads of the stop flag

// scalar slots in d_red after the two partial arrays
enum { S_RZ = 0, S_BB, S_PQ, S_ALPHA, S_BETA, S_REL, S_RR, S_TRUE, kScalars = 16 };
// flags[0]: 0 running, 1 converged, 2 breakdown, 3 NaN/Inf, 4 maxit; flags[1]: iterations
enum { F_STATE = 0, F_ITERS = 1 };
enum { ST_RUN = 0, ST_CONV = 1, ST_BREAK = 2, ST_NAN = 3, ST_MAXIT = 4 };

// Deterministic block sum of two values; thread 0 writes them to part0/part1[blockIdx.x].
__device__ __forceinline__ void block_sum2(double a, double b, double* part0, double* part1) {
  __shared__ double sa[kReduceThreads / 32], sb[kReduceThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  if (l == 0) {
    sa[w] = a;
    sb[w] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0.0, tb = 0.0;
    for (int i = 0; i < kReduceThreads / 32; ++i) {
      ta += sa[i];
      tb += sb[i];
    }
    part0[blockIdx.x] = ta;
    if (part1) part1[blockIdx.x] = tb;
  }
}

__device__ __forceinline__ double ordered_sum(const double* part) {
  double s = 0.0;
  for (int i = 0; i < kReduceBlocks; ++i) s += part[i];
  return s;
}

__global__ void __launch_bounds__(kReduceThreads) k_init(const double* __restrict__ b,
                                                         const uint8_t* __restrict__ mask,
                                                         const double* __restrict__ d,
                                                         double* __restrict__ x,
                                                         double* __restrict__ r,
                                                         double* __restrict__ z,
                                                         double* __restrict__ p, int64_t n,
                                                         double* part0, double* part1) {
  double s_rz = 0.0, s_bb = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double bi = mask[i] ? 0.0 : b[i];
    const double zi = d ? bi / d[i] : bi;
    x[i] = 0.0;
    r[i] = bi;
    z[i] = zi;
    p[i] = zi;
    s_rz = fma(bi, zi, s_rz);
    s_bb = fma(bi, bi, s_bb);
  }
  block_sum2(s_rz, s_bb, part0, part1);
}

__global__ void k_finish_init(const double* part0, const double* part1, double* sc, int* flags) {
  const double rz = ordered_sum(part0), bb = ordered_sum(part1);
  sc[S_RZ] = rz;
  sc[S_BB] = bb;
  sc[S_REL] = 0.0;
  flags[F_ITERS] = 0;
  if (!isfinite(rz) || !isfinite(bb))
    flags[F_STATE] = ST_NAN;
  else if (bb == 0.0)
    flags[F_STATE] = ST_CONV;
  else
    flags[F_STATE] = ST_RUN;
  if (flags[F_STATE] == ST_RUN) sc[S_REL] = 1.0;
}

__global__ void __launch_bounds__(kReduceThreads) k_zero(double* __restrict__ v, int64_t n,
                                                         const int* flags) {
  if (flags[F_STATE] != ST_RUN) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] = 0.0;
}

__global__ void __launch_bounds__(kReduceThreads) k_dot(const double* __restrict__ a,
                                                        const double* __restrict__ b, int64_t n,
                                                        double* part0, const int* flags) {
  if (flags[F_STATE] != ST_RUN) return;
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s = fma(a[i], b[i], s);
  block_sum2(s, 0.0, part0, nullptr);
}

__global__ void k_finish_pq(const double* part0, double* sc, int* flags) {
  if (flags[F_STATE] != ST_RUN) return;
  const double pq = ordered_sum(part0);
  sc[S_PQ] = pq;
  if (!isfinite(pq))
    flags[F_STATE] = ST_NAN;
  else if (!(pq > 0.0))
    flags[F_STATE] = ST_BREAK;
  else
    sc[S_ALPHA] = sc[S_RZ] / pq;
}

__global__ void __launch_bounds__(kReduceThreads) k_update(double* __restrict__ x,
                                                           double* __restrict__ r,
                                                           double* __restrict__ z,
                                                           const double* __restrict__ p,
                                                           const double* __restrict__ q,
                                                           const double* __restrict__ d,
                                                           const uint8_t* __restrict__ mask,
                                                           int64_t n, const double* sc,
                                                           double* part0, double* part1,
                                                           const int* flags) {
  if (flags[F_STATE] != ST_RUN) return;
  const double alpha = sc[S_ALPHA];
  double s_rz = 0.0, s_rr = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const bool bnd = mask[i] != 0;
    const double qi = bnd ? 0.0 : q[i];
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, qi, r[i]);
    r[i] = ri;
    const double zi = bnd ? 0.0 : (d ? ri / d[i] : ri);
    z[i] = zi;
    s_rz = fma(ri, zi, s_rz);
    s_rr = fma(ri, ri, s_rr);
  }
  block_sum2(s_rz, s_rr, part0, part1);
}

__global__ void k_finish_update(const double* part0, const double* part1, double* sc,
                                int* flags, double rtol, int maxit) {
  if (flags[F_STATE] != ST_RUN) return;
  const double rz = ordered_sum(part0), rr = ordered_sum(part1);
  const int it = flags[F_ITERS] + 1;
  flags[F_ITERS] = it;
  const double rel = sqrt(rr / sc[S_BB]);
  sc[S_REL] = rel;
  sc[S_RR] = rr;
  if (!isfinite(rz) || !isfinite(rel)) {
    flags[F_STATE] = ST_NAN;
    return;
  }
  if (rel <= rtol) {
    flags[F_STATE] = ST_CONV;
    return;
  }
  sc[S_BETA] = rz / sc[S_RZ];
  sc[S_RZ] = rz;
  if (it >= maxit) flags[F_STATE] = ST_MAXIT;
}

__global__ void __launch_bounds__(kReduceThreads) k_pupdate(double* __restrict__ p,
                                                            const double* __restrict__ z,
                                                            int64_t n, const double* sc,
                                                            const int* flags) {
  if (flags[F_STATE] != ST_RUN) return;
  const double beta = sc[S_BETA];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = fma(beta, p[i], z[i]);
}

// Jacobi: boundary entries of the diagonal set to 1 (they are never used); any non-positive
// interior entry is reported through flags as a breakdown.
__global__ void __launch_bounds__(kReduceThreads) k_fix_diag(double* __restrict__ d,
                                                             const uint8_t* __restrict__ mask,
                                                             int64_t n, int* flags) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (mask[i])
      d[i] = 1.0;
    else if (!(d[i] > 0.0))
      atomicExch(&flags[2], 1);
  }
}

// ||(1-m)(b - q)||^2 partials for the true residual.
__global__ void __launch_bounds__(kReduceThreads) k_resid(const double* __restrict__ b,
                                                          const double* __restrict__ q,
                                                          const uint8_t* __restrict__ mask,
                                                          int64_t n, double* part0) {
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = mask[i] ? 0.0 : b[i] - q[i];
    s = fma(ri, ri, s);
  }
  block_sum2(s, 0.0, part0, nullptr);
}

__global__ void k_finish_resid(const double* part0, double* sc) {
  sc[S_TRUE] = sqrt(ordered_sum(part0) / sc[S_BB]);
}

}  // namespace

extern "C" int fe_pcg(fe_pa* pa, int op, int pc, const double* dev_b, double* dev_x, double rtol,
                      int maxit, fe_pcg_stats* stats, void* stream) {
  clear_error();
  const auto t0 = std::chrono::steady_clock::now();
  if (stats) *stats = fe_pcg_stats{0, 0.0, 0.0, 0.0, 0};
  int launches = 0;
  if (!pa || !dev_b || !dev_x) return set_error(FE_ERR_ARG, "fe_pcg: null argument");
  if (op != FE_DIFFUSION && op != FE_MASS) return set_error(FE_ERR_ARG, "fe_pcg: bad op");
  if (!(pa->ops & op)) return set_error(FE_ERR_ARG, "fe_pcg: operator not set up");
  if (pc != FE_PC_NONE && pc != FE_PC_JACOBI) return set_error(FE_ERR_ARG, "fe_pcg: bad preconditioner");
  if (maxit < 1 || !(rtol >= 0.0)) return set_error(FE_ERR_ARG, "fe_pcg: bad rtol or maxit");
  cudaStream_t s = (cudaStream_t)stream;
  const fe_mesh* m = pa->mesh;
  const int64_t n = m->ndofs;
  cudaError_t err;
  if (pa->work_ndofs != n) {
    cudaFree(pa->d_work);
    cudaFree(pa->d_red);
    cudaFree(pa->d_flags);
    pa->d_work = pa->d_red = nullptr;
    pa->d_flags = nullptr;
    pa->work_ndofs = 0;
    if ((err = cudaMalloc(&pa->d_work, sizeof(double) * 5 * n)) != cudaSuccess ||
        (err = cudaMalloc(&pa->d_red, sizeof(double) * (2 * kReduceBlocks + kScalars))) !=
            cudaSuccess ||
        (err = cudaMalloc(&pa->d_flags, sizeof(int) * 4)) != cudaSuccess)
      return cuda_error(err, "fe_pcg: workspace cudaMalloc");
    pa->work_ndofs = n;
  }
  double* r = pa->d_work;
  double* z = r + n;
  double* p = z + n;
  double* q = p + n;
  double* d = q + n;
  double* part0 = pa->d_red;
  double* part1 = part0 + kReduceBlocks;
  double* sc = part1 + kReduceBlocks;
  int* flags = pa->d_flags;
  const uint8_t* mask = m->d_mask;

#define PCG_LAUNCH_CHECK(what)                                  \
  do {                                                          \
    cudaError_t e_ = cudaGetLastError();                        \
    if (e_ != cudaSuccess) return cuda_error(e_, what);         \
  } while (0)


  if ((err = cudaMemsetAsync(flags, 0, sizeof(int) * 4, s)) != cudaSuccess)
    return cuda_error(err, "fe_pcg: flags");
  const double* dj = nullptr;
  if (pc == FE_PC_JACOBI) {
    int st = fe_assemble_diagonal(pa, op, d, stream);
    if (st != FE_OK) return st;
    k_fix_diag<<<kReduceBlocks, kReduceThreads, 0, s>>>(d, mask, n, flags);
    PCG_LAUNCH_CHECK("fe_pcg: diag fix launch");
    launches += 2;
    dj = d;
  }
  k_init<<<kReduceBlocks, kReduceThreads, 0, s>>>(dev_b, mask, dj, dev_x, r, z, p, n, part0, part1);
  k_finish_init<<<1, 1, 0, s>>>(part0, part1, sc, flags);
  PCG_LAUNCH_CHECK("fe_pcg: init launch");
  launches += 2;
  int hflags[4] = {0, 0, 0, 0};
  if (pc == FE_PC_JACOBI) {
    if ((err = cudaMemcpyAsync(hflags, flags, sizeof(int) * 4, cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess ||
        (err = cudaStreamSynchronize(s)) != cudaSuccess)
      return cuda_error(err, "fe_pcg: init");
    if (hflags[2]) return set_error(FE_ERR_BREAKDOWN, "fe_pcg: non-positive diagonal entry");
  }
  int queued = 0;
  for (;;) {
    for (int j = 0; j < kBatch && queued < maxit; ++j, ++queued) {
      k_zero<<<kReduceBlocks, kReduceThreads, 0, s>>>(q, n, flags);
      int st = apply_dispatch(pa, op, pa->variant, p, q, s, flags);
      if (st != FE_OK) return st;
      k_dot<<<kReduceBlocks, kReduceThreads, 0, s>>>(p, q, n, part0, flags);
      k_finish_pq<<<1, 1, 0, s>>>(part0, sc, flags);
      k_update<<<kReduceBlocks, kReduceThreads, 0, s>>>(dev_x, r, z, p, q, dj, mask, n, sc, part0,
                                                          part1, flags);
      k_finish_update<<<1, 1, 0, s>>>(part0, part1, sc, flags, rtol, maxit);
      k_pupdate<<<kReduceBlocks, kReduceThreads, 0, s>>>(p, z, n, sc, flags);
      PCG_LAUNCH_CHECK("fe_pcg: iteration launch");
      launches += 7;
    }
    if ((err = cudaMemcpyAsync(hflags, flags, sizeof(int) * 4, cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess ||
        (err = cudaStreamSynchronize(s)) != cudaSuccess)
      return cuda_error(err, "fe_pcg: iteration");
    if (hflags[F_STATE] != ST_RUN || queued >= maxit) break;
  }
  // true residual ||(1-m)(b - A x)|| / ||b|| with the same apply
  int st = apply_dispatch(pa, op, pa->variant, dev_x, q, s);
  if (st != FE_OK) return st;
  k_resid<<<kReduceBlocks, kReduceThreads, 0, s>>>(dev_b, q, mask, n, part0);
  k_finish_resid<<<1, 1, 0, s>>>(part0, sc);
  PCG_LAUNCH_CHECK("fe_pcg: residual launch");
  launches += 3;
  double hsc[kScalars];
  if ((err = cudaMemcpyAsync(hsc, sc, sizeof(double) * kScalars, cudaMemcpyDeviceToHost, s)) !=
          cudaSuccess ||
      (err = cudaStreamSynchronize(s)) != cudaSuccess)
    return cuda_error(err, "fe_pcg: stats");
#undef PCG_LAUNCH_CHECK
  if (stats) {
    stats->iters = hflags[F_ITERS];
    stats->rel_resid = hsc[S_REL];
    stats->true_rel_resid = hsc[S_BB] > 0.0 ? hsc[S_TRUE] : 0.0;
    stats->seconds =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    stats->launches = launches;
  }
  switch (hflags[F_STATE]) {
    case ST_CONV:
      return FE_OK;
    case ST_BREAK:
      return set_error(FE_ERR_BREAKDOWN, "fe_pcg: p.Ap <= 0 (operator not SPD on the free dofs)");
    case ST_NAN:
      return set_error(FE_ERR_NAN, "fe_pcg: NaN or Inf in the iteration");
    default:
      return set_error(FE_ERR_NOT_CONVERGED, "fe_pcg: maxit reached before rtol");
  }
}

// ------------------------------------------------------------------------------------------
// fe_pcg_noalloc: the same Jacobi-PCG for callers that must not allocate device memory.
//
// Some callers cannot let a library call cudaMalloc: applications that hand (nearly) all of
// the GPU's memory to their own pool allocator up front, so that a driver allocation would fail
// or fragment the pool, and latency-critical loops that cannot afford the blocking and device
// synchronisation that cudaMalloc and cudaFree can cause.  This entry point therefore takes its
// work vectors, reduction partials and flags from one fixed device array that is part of the
// library image (kNoAllocMaxDofs dofs; about 10.5 MB, held on every GPU that loads the
// library until the process exits) instead of allocating them.
namespace {

constexpr int64_t kNoAllocMaxDofs = (int64_t)1 << 18;  // 262,144 dofs, e.g. 64^3 GLL points
constexpr int64_t kNoAllocDoubles =
    5 * kNoAllocMaxDofs + 2 * kReduceBlocks + kScalars + 2;  // + 4 ints of flags

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

// Device address of g_noalloc_scratch per device, looked up once with that device current.
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[64] = {nullptr};

int noalloc_scratch(double** out) {
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return cuda_error(err, "fe_pcg_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= 64) return set_error(FE_ERR_UNSUPPORTED, "fe_pcg_noalloc: device index >= 64");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* p = nullptr;
    err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (err != cudaSuccess) return cuda_error(err, "fe_pcg_noalloc: cudaGetSymbolAddress");
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return FE_OK;
}

}  // namespace

extern "C" int fe_pcg_noalloc(const fe_pa* pa, int op, int pc, const double* dev_b,
                              double* dev_x, double rtol, int maxit, fe_pcg_stats* stats,
                              void* stream) {
  clear_error();
  const auto t0 = std::chrono::steady_clock::now();
  if (stats) *stats = fe_pcg_stats{0, 0.0, 0.0, 0.0, 0};
  int launches = 0;
  if (!pa || !dev_b || !dev_x) return set_error(FE_ERR_ARG, "fe_pcg_noalloc: null argument");
  if (op != FE_DIFFUSION && op != FE_MASS) return set_error(FE_ERR_ARG, "fe_pcg_noalloc: bad op");
  if (!(pa->ops & op)) return set_error(FE_ERR_ARG, "fe_pcg_noalloc: operator not set up");
  if (pc != FE_PC_NONE && pc != FE_PC_JACOBI)
    return set_error(FE_ERR_ARG, "fe_pcg_noalloc: bad preconditioner");
  if (maxit < 1 || !(rtol >= 0.0)) return set_error(FE_ERR_ARG, "fe_pcg_noalloc: bad rtol or maxit");
  const fe_mesh* m = pa->mesh;
  const int64_t n = m->ndofs;
  if (n > kNoAllocMaxDofs)
    return set_error(FE_ERR_ARG, "fe_pcg_noalloc: the mesh has " + std::to_string(n) +
                                     " dofs, more than the fixed scratch holds (" +
                                     std::to_string(kNoAllocMaxDofs) + "); use fe_pcg");
  double* base = nullptr;
  int st = noalloc_scratch(&base);
  if (st != FE_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  double* r = base;
  double* z = r + n;
  double* p = z + n;
  double* q = p + n;
  double* d = q + n;
  double* part0 = base + 5 * kNoAllocMaxDofs;
  double* part1 = part0 + kReduceBlocks;
  double* sc = part1 + kReduceBlocks;
  int* flags = reinterpret_cast<int*>(sc + kScalars);
  const uint8_t* mask = m->d_mask;
  cudaError_t err;

#define NOALLOC_LAUNCH_CHECK(what)                              \
  do {                                                          \
    cudaError_t e_ = cudaGetLastError();                        \
    if (e_ != cudaSuccess) return cuda_error(e_, what);         \
  } while (0)

  // the array keeps the previous call's contents: the flags must start at zero; every vector
  // and partial is written before it is read (d by the diagonal assembly, q by k_zero)
  if ((err = cudaMemsetAsync(flags, 0, sizeof(int) * 4, s)) != cudaSuccess)
    return cuda_error(err, "fe_pcg_noalloc: flags");
  const double* dj = nullptr;
  if (pc == FE_PC_JACOBI) {
    st = fe_assemble_diagonal(pa, op, d, stream);
    if (st != FE_OK) return st;
    k_fix_diag<<<kReduceBlocks, kReduceThreads, 0, s>>>(d, mask, n, flags);
    NOALLOC_LAUNCH_CHECK("fe_pcg_noalloc: diag fix launch");
    launches += 2;
    dj = d;
  }
  k_init<<<kReduceBlocks, kReduceThreads, 0, s>>>(dev_b, mask, dj, dev_x, r, z, p, n, part0, part1);
  k_finish_init<<<1, 1, 0, s>>>(part0, part1, sc, flags);
  NOALLOC_LAUNCH_CHECK("fe_pcg_noalloc: init launch");
  launches += 2;
  int hflags[4] = {0, 0, 0, 0};
  if (pc == FE_PC_JACOBI) {
    if ((err = cudaMemcpyAsync(hflags, flags, sizeof(int) * 4, cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess ||
        (err = cudaStreamSynchronize(s)) != cudaSuccess)
      return cuda_error(err, "fe_pcg_noalloc: init");
    if (hflags[2]) return set_error(FE_ERR_BREAKDOWN, "fe_pcg_noalloc: non-positive diagonal entry");
  }
  int queued = 0;
  for (;;) {
    for (int j = 0; j < kBatch && queued < maxit; ++j, ++queued) {
      k_zero<<<kReduceBlocks, kReduceThreads, 0, s>>>(q, n, flags);
      st = apply_dispatch(pa, op, pa->variant, p, q, s, flags);
      if (st != FE_OK) return st;
      k_dot<<<kReduceBlocks, kReduceThreads, 0, s>>>(p, q, n, part0, flags);
      k_finish_pq<<<1, 1, 0, s>>>(part0, sc, flags);
      k_update<<<kReduceBlocks, kReduceThreads, 0, s>>>(dev_x, r, z, p, q, dj, mask, n, sc, part0,
                                                          part1, flags);
      k_finish_update<<<1, 1, 0, s>>>(part0, part1, sc, flags, rtol, maxit);
      k_pupdate<<<kReduceBlocks, kReduceThreads, 0, s>>>(p, z, n, sc, flags);
      NOALLOC_LAUNCH_CHECK("fe_pcg_noalloc: iteration launch");
      launches += 7;
    }
    if ((err = cudaMemcpyAsync(hflags, flags, sizeof(int) * 4, cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess ||
        (err = cudaStreamSynchronize(s)) != cudaSuccess)
      return cuda_error(err, "fe_pcg_noalloc: iteration");
    if (hflags[F_STATE] != ST_RUN || queued >= maxit) break;
  }
  st = apply_dispatch(pa, op, pa->variant, dev_x, q, s);
  if (st != FE_OK) return st;
  k_resid<<<kReduceBlocks, kReduceThreads, 0, s>>>(dev_b, q, mask, n, part0);
  k_finish_resid<<<1, 1, 0, s>>>(part0, sc);
  NOALLOC_LAUNCH_CHECK("fe_pcg_noalloc: residual launch");
  launches += 3;
  double hsc[kScalars];
  if ((err = cudaMemcpyAsync(hsc, sc, sizeof(double) * kScalars, cudaMemcpyDeviceToHost, s)) !=
          cudaSuccess ||
      (err = cudaStreamSynchronize(s)) != cudaSuccess)
    return cuda_error(err, "fe_pcg_noalloc: stats");
#undef NOALLOC_LAUNCH_CHECK
  if (stats) {
    stats->iters = hflags[F_ITERS];
    stats->rel_resid = hsc[S_REL];
    stats->true_rel_resid = hsc[S_BB] > 0.0 ? hsc[S_TRUE] : 0.0;
    stats->seconds =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    stats->launches = launches;
  }
  switch (hflags[F_STATE]) {
    case ST_CONV:
      return FE_OK;
    case ST_BREAK:
      return set_error(FE_ERR_BREAKDOWN, "fe_pcg_noalloc: p.Ap <= 0 (operator not SPD on the free dofs)");
    case ST_NAN:
      return set_error(FE_ERR_NAN, "fe_pcg_noalloc: NaN or Inf in the iteration");
    default:
      return set_error(FE_ERR_NOT_CONVERGED, "fe_pcg_noalloc: maxit reached before rtol");
  }
}
