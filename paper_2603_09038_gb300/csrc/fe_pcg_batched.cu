// Batched Jacobi-PCG: nrhs independent systems A_bc x_j = b_j with one operator, advanced in
// lockstep so that every iteration applies the operator to all search directions in ONE batched
// launch (each block applies all right-hand sides to its elements, reading its dof map and
// quadrature data once from HBM and then from L2).  Every right-hand side keeps its own scalars,
// stop state and iteration count on the device; a system that has converged (or broken down)
// stops updating while the others go on, and the batch ends when all have stopped.  The vector
// kernels run on a 2D grid (blocks x right-hand sides) with the same deterministic reductions as
// fe_pcg, and iteration batches are replayed as CUDA graphs.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <string>
#include <vector>

#include "fe_f2.h"
#include "fe_internal.h"

namespace {

using namespace fe;

#include "fe_solver_common.cuh"

// ctl[0]: systems still running; ctl[1]: 1 once none is (the apply's skip flag)
enum { C_RUNNING = 0, C_DONE = 1 };

__device__ __forceinline__ void stop(int* flags, int state, int* ctl) {
  flags[F_STATE] = state;
  if (atomicSub(&ctl[C_RUNNING], 1) == 1) ctl[C_DONE] = 1;
}

// r = (1-m) b, z = dinv r (or r), p = z, q = 0, x = 0; r.z and b.b partials
__global__ void __launch_bounds__(kReduceThreads) k_binit(const double* __restrict__ B, int64_t ldb,
                                                          const uint8_t* __restrict__ mask,
                                                          const double* __restrict__ dinv,
                                                          double* __restrict__ X, int64_t ldx,
                                                          double* __restrict__ R,
                                                          double* __restrict__ Z,
                                                          double* __restrict__ P,
                                                          double* __restrict__ Q, int64_t n,
                                                          double* part0, double* part1) {
  const int j = blockIdx.y;
  const double* b = B + j * ldb;
  double* x = X + j * ldx;
  double *r = R + j * n, *z = Z + j * n, *p = P + j * n, *q = Q + j * n;
  double s_rz = 0.0, s_bb = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double bi = mask[i] ? 0.0 : b[i];
    const double zi = dinv ? bi * dinv[i] : bi;
    x[i] = 0.0;
    r[i] = bi;
    z[i] = zi;
    p[i] = zi;
    q[i] = 0.0;
    s_rz = fma(bi, zi, s_rz);
    s_bb = fma(bi, bi, s_bb);
  }
  block_sum2(s_rz, s_bb, part0 + j * kReduceBlocks, part1 + j * kReduceBlocks);
}

__global__ void __launch_bounds__(kFinishThreads) k_bfinish_init(const double* part0,
                                                               const double* part1, double* sc,
                                                               int* flags, int* ctl) {
  const int j = blockIdx.x;
  const double rz = ordered_sum(part0 + j * kReduceBlocks);
  const double bb = ordered_sum(part1 + j * kReduceBlocks);
  if (threadIdx.x != 0) return;
  double* s = sc + j * kScalars;
  int* f = flags + j * 4;
  s[S_RZ] = rz;
  s[S_BB] = bb;
  s[S_REL] = 0.0;
  f[F_ITERS] = 0;
  if (!isfinite(rz) || !isfinite(bb)) {
    f[F_STATE] = ST_NAN;
  } else if (bb == 0.0) {
    f[F_STATE] = ST_CONV;
  } else {
    f[F_STATE] = ST_RUN;
    s[S_REL] = 1.0;
    atomicAdd(&ctl[C_RUNNING], 1);
  }
}

// after all systems' init: done when none runs
__global__ void k_bcheck(int* ctl) {
  if (threadIdx.x == 0 && ctl[C_RUNNING] == 0) ctl[C_DONE] = 1;
}

__global__ void __launch_bounds__(kReduceThreads) k_bdot(const double* __restrict__ P,
                                                         const double* __restrict__ Q, int64_t n,
                                                         double* part0, const int* flags) {
  const int j = blockIdx.y;
  if (flags[j * 4 + F_STATE] != ST_RUN) return;
  const double *p = P + j * n, *q = Q + j * n;
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s = fma(p[i], q[i], s);
  block_sum2(s, 0.0, part0 + j * kReduceBlocks, nullptr);
}

__global__ void __launch_bounds__(kFinishThreads) k_bfinish_pq(const double* part0, double* sc,
                                                             int* flags, int* ctl) {
  const int j = blockIdx.x;
  int* f = flags + j * 4;
  if (f[F_STATE] != ST_RUN) return;
  const double pq = ordered_sum(part0 + j * kReduceBlocks);
  if (threadIdx.x != 0) return;
  double* s = sc + j * kScalars;
  s[S_PQ] = pq;
  if (!isfinite(pq))
    stop(f, ST_NAN, ctl);
  else if (!(pq > 0.0))
    stop(f, ST_BREAK, ctl);
  else
    s[S_ALPHA] = s[S_RZ] / pq;
}

__global__ void __launch_bounds__(kReduceThreads) k_bupdate(double* __restrict__ X, int64_t ldx,
                                                            double* __restrict__ R,
                                                            double* __restrict__ Z,
                                                            const double* __restrict__ P,
                                                            const double* __restrict__ Q,
                                                            const double* __restrict__ dinv,
                                                            const uint8_t* __restrict__ mask,
                                                            int64_t n, const double* sc,
                                                            double* part0, double* part1,
                                                            const int* flags) {
  const int j = blockIdx.y;
  if (flags[j * 4 + F_STATE] != ST_RUN) return;
  const double alpha = sc[j * kScalars + S_ALPHA];
  double* x = X + j * ldx;
  double *r = R + j * n, *z = Z + j * n;
  const double *p = P + j * n, *q = Q + j * n;
  double s_rz = 0.0, s_rr = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const bool bnd = mask[i] != 0;
    const double qi = bnd ? 0.0 : q[i];
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, qi, r[i]);
    r[i] = ri;
    const double zi = dinv ? ri * dinv[i] : (bnd ? 0.0 : ri);
    z[i] = zi;
    s_rz = fma(ri, zi, s_rz);
    s_rr = fma(ri, ri, s_rr);
  }
  block_sum2(s_rz, s_rr, part0 + j * kReduceBlocks, part1 + j * kReduceBlocks);
}

__global__ void __launch_bounds__(kFinishThreads) k_bfinish_update(const double* part0,
                                                                 const double* part1, double* sc,
                                                                 int* flags, int* ctl,
                                                                 double rtol, int maxit) {
  const int j = blockIdx.x;
  int* f = flags + j * 4;
  if (f[F_STATE] != ST_RUN) return;
  const double rz = ordered_sum(part0 + j * kReduceBlocks);
  const double rr = ordered_sum(part1 + j * kReduceBlocks);
  if (threadIdx.x != 0) return;
  double* s = sc + j * kScalars;
  const int it = f[F_ITERS] + 1;
  f[F_ITERS] = it;
  const double rel = sqrt(rr / s[S_BB]);
  s[S_REL] = rel;
  if (!isfinite(rz) || !isfinite(rel)) {
    stop(f, ST_NAN, ctl);
    return;
  }
  if (rel <= rtol) {
    stop(f, ST_CONV, ctl);
    return;
  }
  s[S_BETA] = rz / s[S_RZ];
  s[S_RZ] = rz;
  if (it >= maxit) stop(f, ST_MAXIT, ctl);
}

// p = z + beta p for the running systems; q = 0 for all (the next batched apply adds into it)
__global__ void __launch_bounds__(kReduceThreads) k_bpupdate(double* __restrict__ P,
                                                             const double* __restrict__ Z,
                                                             double* __restrict__ Q, int64_t n,
                                                             const double* sc, const int* flags,
                                                             const int* ctl) {
  if (ctl[C_DONE]) return;
  const int j = blockIdx.y;
  const bool run = flags[j * 4 + F_STATE] == ST_RUN;
  const double beta = sc[j * kScalars + S_BETA];
  double* p = P + j * n;
  const double* z = Z + j * n;
  double* q = Q + j * n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (run) p[i] = fma(beta, p[i], z[i]);
    q[i] = 0.0;
  }
}

// ||(1-m)(b - A x)||^2 and ||(1-m) b||^2 partials per system (Q = A X)
__global__ void __launch_bounds__(kReduceThreads) k_bresid(const double* __restrict__ B,
                                                           int64_t ldb,
                                                           const double* __restrict__ Q,
                                                           const uint8_t* __restrict__ mask,
                                                           int64_t n, double* part0,
                                                           double* part1) {
  const int j = blockIdx.y;
  const double* b = B + j * ldb;
  const double* q = Q + j * n;
  double s = 0.0, sb = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (mask[i]) continue;
    const double d = b[i] - q[i];
    s = fma(d, d, s);
    sb = fma(b[i], b[i], sb);
  }
  block_sum2(s, sb, part0 + j * kReduceBlocks, part1 + j * kReduceBlocks);
}

__global__ void __launch_bounds__(kFinishThreads) k_bfinish_resid(const double* part0,
                                                                const double* part1,
                                                                double* sc) {
  const int j = blockIdx.x;
  const double rr = ordered_sum(part0 + j * kReduceBlocks);
  const double bb = ordered_sum(part1 + j * kReduceBlocks);
  if (threadIdx.x == 0) sc[j * kScalars + S_TRUE] = bb > 0.0 ? sqrt(rr / bb) : 0.0;
}

__global__ void k_invert_diag_b(double* __restrict__ d, const uint8_t* __restrict__ mask,
                                int64_t n, int* bad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (mask[i]) {
      d[i] = 0.0;
    } else {
      const double di = d[i];
      if (!(di > 0.0)) atomicExch(bad, 1);
      d[i] = 1.0 / di;
    }
  }
}

struct Buffers {
  double* vec = nullptr;  // R, Z, P, Q (nrhs x n each), dinv (n)
  double* red = nullptr;  // partials (2 x nrhs x kReduceBlocks), scalars (nrhs x kScalars)
  int* flags = nullptr;   // nrhs x 4, then ctl[2], then a breakdown flag
  ~Buffers() {
    cudaFree(vec);
    cudaFree(red);
    cudaFree(flags);
  }
};

}  // namespace

namespace fe {

// The lockstep batched Jacobi- (or un-) preconditioned CG of fe_pcg_batched around any operator
// (see BatchedOperator in fe_internal.h).
int pcg_batched_core(const BatchedOperator& A, int nrhs, const double* dev_b, int64_t ldb,
                     double* dev_x, int64_t ldx, double rtol, int maxit, fe_pcg_stats* stats,
                     cudaStream_t s, const char* who) {
  const auto t0 = std::chrono::steady_clock::now();
  const std::string w(who);
  const int64_t n = A.n;
  if (nrhs < 1 || nrhs > 1024 || ldb < n || ldx < n)
    return set_error(FE_ERR_ARG, w + ": need 1 <= nrhs <= 1024 and ldb, ldx >= ndofs");
  if (maxit < 1 || !(rtol >= 0.0)) return set_error(FE_ERR_ARG, w + ": bad rtol or maxit");
  if (stats)
    for (int j = 0; j < nrhs; ++j) stats[j] = fe_pcg_stats{0, 0.0, 0.0, 0.0, 0, 0};
  Buffers buf;
  cudaError_t err;
  const size_t nv = (size_t)nrhs * n;
  if ((err = cudaMalloc(&buf.vec, sizeof(double) * (4 * nv + n))) != cudaSuccess ||
      (err = cudaMalloc(&buf.red, sizeof(double) * ((size_t)2 * nrhs * kReduceBlocks +
                                                    (size_t)nrhs * kScalars))) != cudaSuccess ||
      (err = cudaMalloc(&buf.flags, sizeof(int) * (4 * nrhs + 3))) != cudaSuccess)
    return cuda_error(err, (w + ": cudaMalloc").c_str());
  double *R = buf.vec, *Z = R + nv, *P = Z + nv, *Q = P + nv, *dinv = Q + nv;
  double *part0 = buf.red, *part1 = part0 + (size_t)nrhs * kReduceBlocks,
         *sc = part1 + (size_t)nrhs * kReduceBlocks;
  int* flags = buf.flags;
  int* ctl = flags + 4 * nrhs;
  int* bad = ctl + 2;
  int launches = 0;
  if ((err = cudaMemsetAsync(flags, 0, sizeof(int) * (4 * nrhs + 3), s)) != cudaSuccess)
    return cuda_error(err, (w + ": flags").c_str());
  int st = FE_OK;
  if (A.diagonal) {
    if ((st = A.diagonal(s, dinv)) != FE_OK) return st;
    k_invert_diag_b<<<kReduceBlocks, kReduceThreads, 0, s>>>(dinv, A.mask, n, bad);
    launches += 2;
  }
  const double* dj = A.diagonal ? dinv : nullptr;
  const dim3 grid2(kReduceBlocks, nrhs);
  k_binit<<<grid2, kReduceThreads, 0, s>>>(dev_b, ldb, A.mask, dj, dev_x, ldx, R, Z, P, Q, n,
                                           part0, part1);
  k_bfinish_init<<<nrhs, kFinishThreads, 0, s>>>(part0, part1, sc, flags, ctl);
  k_bcheck<<<1, 32, 0, s>>>(ctl);
  launches += 3;
  if ((err = cudaGetLastError()) != cudaSuccess) return cuda_error(err, (w + ": init").c_str());
  auto enqueue = [&](cudaStream_t q, int count, int* nk) -> int {
    for (int it = 0; it < count; ++it) {
      int st2 = A.apply(q, nrhs, P, Q, ctl + C_DONE, nk);
      if (st2 != FE_OK) return st2;
      k_bdot<<<grid2, kReduceThreads, 0, q>>>(P, Q, n, part0, flags);
      k_bfinish_pq<<<nrhs, kFinishThreads, 0, q>>>(part0, sc, flags, ctl);
      k_bupdate<<<grid2, kReduceThreads, 0, q>>>(dev_x, ldx, R, Z, P, Q, dj, A.mask, n, sc,
                                                 part0, part1, flags);
      k_bfinish_update<<<nrhs, kFinishThreads, 0, q>>>(part0, part1, sc, flags, ctl, rtol, maxit);
      k_bpupdate<<<grid2, kReduceThreads, 0, q>>>(P, Z, Q, n, sc, flags, ctl);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_error(e, (w + ": iteration launch").c_str());
      *nk += 5;
    }
    return FE_OK;
  };
  int hctl[3] = {0, 0, 0};
  int queued = 0;
  GraphBatch graph;
  for (;;) {
    if ((err = cudaMemcpyAsync(hctl, ctl, sizeof(int) * 3, cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess ||
        (err = cudaStreamSynchronize(s)) != cudaSuccess)
      return cuda_error(err, (w + ": iteration").c_str());
    if (hctl[2]) return set_error(FE_ERR_BREAKDOWN, w + ": non-positive diagonal entry");
    if (hctl[C_DONE] || queued >= maxit) break;
    const int count = maxit - queued < kBatch ? maxit - queued : kBatch;
    if (queued > 0 && count == kBatch && A.graphs && !graph.failed && !graph.exec) {
      int nk = 0;
      graph.capture([&](cudaStream_t q) { return enqueue(q, kBatch, &nk); });
      graph.kernels = nk;
    }
    if (graph.exec && count == kBatch) {
      if ((err = cudaGraphLaunch(graph.exec, s)) != cudaSuccess)
        return cuda_error(err, (w + ": graph launch").c_str());
      launches += graph.kernels;
    } else if ((st = enqueue(s, count, &launches)) != FE_OK) {
      return st;
    }
    queued += count;
  }
  // true residuals with the FP64 operator: Q = A X, per-system norms
  if ((st = A.apply_fp64(s, nrhs, dev_x, ldx, Q, &launches)) != FE_OK) return st;
  k_bresid<<<grid2, kReduceThreads, 0, s>>>(dev_b, ldb, Q, A.mask, n, part0, part1);
  k_bfinish_resid<<<nrhs, kFinishThreads, 0, s>>>(part0, part1, sc);
  launches += 2;
  std::vector<double> hsc((size_t)nrhs * kScalars);
  std::vector<int> hf((size_t)nrhs * 4);
  if ((err = cudaGetLastError()) != cudaSuccess ||
      (err = cudaMemcpyAsync(hsc.data(), sc, sizeof(double) * hsc.size(), cudaMemcpyDeviceToHost,
                             s)) != cudaSuccess ||
      (err = cudaMemcpyAsync(hf.data(), flags, sizeof(int) * hf.size(), cudaMemcpyDeviceToHost,
                             s)) != cudaSuccess ||
      (err = cudaStreamSynchronize(s)) != cudaSuccess)
    return cuda_error(err, (w + ": stats").c_str());
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  int worst = FE_OK;
  for (int j = 0; j < nrhs; ++j) {
    const int state = hf[j * 4 + F_STATE];
    if (stats) {
      stats[j].iters = hf[j * 4 + F_ITERS];
      stats[j].rel_resid = hsc[j * kScalars + S_REL];
      stats[j].true_rel_resid = hsc[j * kScalars + S_TRUE];
      stats[j].seconds = secs;
      stats[j].launches = launches;
      stats[j].outer_iters = 1;
    }
    int code = FE_OK;
    if (state == ST_BREAK) code = FE_ERR_BREAKDOWN;
    else if (state == ST_NAN) code = FE_ERR_NAN;
    else if (state != ST_CONV) code = FE_ERR_NOT_CONVERGED;
    if (worst == FE_OK && code != FE_OK) worst = code;
  }
  if (worst != FE_OK) return set_error(worst, w + ": some right-hand side did not converge (see stats)");
  return FE_OK;
}

}  // namespace fe

extern "C" int fe_pcg_batched(fe_pa* pa, int op, int pc, int nrhs, const double* dev_b,
                              int64_t ldb, double* dev_x, int64_t ldx, double rtol, int maxit,
                              fe_pcg_stats* stats, void* stream) {
  clear_error();
  if (!pa || !dev_b || !dev_x) return set_error(FE_ERR_ARG, "fe_pcg_batched: null argument");
  if (op != FE_DIFFUSION && op != FE_MASS) return set_error(FE_ERR_ARG, "fe_pcg_batched: bad op");
  if (!(pa->ops & op)) return set_error(FE_ERR_ARG, "fe_pcg_batched: operator not set up");
  if (pc != FE_PC_NONE && pc != FE_PC_JACOBI)
    return set_error(FE_ERR_ARG, "fe_pcg_batched: preconditioner must be none or Jacobi");
  if (pa->variant == FE_VARIANT_F32)
    return set_error(FE_ERR_UNSUPPORTED, "fe_pcg_batched: the FP32 variant is not FP64-accurate");
  const int variant = pa->variant;
  const int64_t n = pa->mesh->ndofs;
  BatchedOperator A;
  A.n = n;
  A.mask = pa->mesh->d_mask;
  A.graphs = pa->pcg_graphs;
  // one batched launch for all search directions (the DMMA kernel applies them one by one)
  A.apply = [=](cudaStream_t q, int nr, const double* P, double* Q, const int* skip,
                int* nk) -> int {
    if (variant != FE_VARIANT_F64_DMMA) {
      ++*nk;
      return apply_dispatch(pa, op, variant, P, Q, q, skip, nullptr, nullptr, false, nr, n, n);
    }
    for (int j = 0; j < nr; ++j) {
      const int st2 = apply_dispatch(pa, op, variant, P + j * n, Q + j * n, q, skip);
      if (st2 != FE_OK) return st2;
      ++*nk;
    }
    return FE_OK;
  };
  A.apply_fp64 = [=](cudaStream_t q, int nr, const double* X, int64_t lx, double* Q,
                     int* nk) -> int {
    ++*nk;
    return apply_dispatch(pa, op, FE_VARIANT_F64, X, Q, q, nullptr, nullptr, nullptr, false, nr,
                          lx, n);
  };
  if (pc == FE_PC_JACOBI)
    A.diagonal = [=](cudaStream_t q, double* d) { return fe_assemble_diagonal(pa, op, d, q); };
  return pcg_batched_core(A, nrhs, dev_b, ldb, dev_x, ldx, rtol, maxit, stats,
                          (cudaStream_t)stream, "fe_pcg_batched");
}
