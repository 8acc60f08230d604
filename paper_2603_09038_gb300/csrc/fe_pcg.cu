// Jacobi-preconditioned conjugate gradients with a device-resident state.
//
// The paper has no solver for this operator (it time-steps a wave equation); fe_pcg is the
// standard preconditioned CG (Hestenes-Stiefel) around the fused apply, with the Dirichlet
// boundary handled by the constrained operator A_bc = (1-m) A (1-m) + m.  Started from zero with
// the boundary entries of b ignored, every iterate, residual and search direction stays zero on
// the boundary, so A_bc p reduces to (1-m) A p.
//
// GB300 layout of one iteration (no host round trip): fused apply q = A p | p.q partials |
// control (alpha) | x, r, z update + r.z, r.r partials | control (beta, stop test) | p update
// (which also zeroes q for the next atomic scatter).  Scalars and the stop flag live in device memory; every kernel returns at once when
// the flag is set, so the host queues iterations in batches and reads the flag once per batch.
// Inner products are deterministic: a fixed grid of kReduceBlocks blocks, fixed in-block trees,
// and the partials summed in block order by a single thread.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "fe_f2.h"
#include "fe_internal.h"

namespace {

using namespace fe;

#include "fe_solver_common.cuh"

__global__ void __launch_bounds__(kReduceThreads) k_init(const double* __restrict__ b,
                                                         const uint8_t* __restrict__ mask,
                                                         const double* __restrict__ d,
                                                         double* __restrict__ x,
                                                         double* __restrict__ r,
                                                         double* __restrict__ z,
                                                         double* __restrict__ p,
                                                         double* __restrict__ q, int64_t n,
                                                         double* part0, double* part1) {
  double s_rz = 0.0, s_bb = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double bi = mask[i] ? 0.0 : b[i];
    const double zi = d ? bi * d[i] : bi;
    x[i] = 0.0;
    r[i] = bi;
    z[i] = zi;
    p[i] = zi;
    q[i] = 0.0;
    s_rz = fma(bi, zi, s_rz);
    s_bb = fma(bi, bi, s_bb);
  }
  block_sum2(s_rz, s_bb, part0, part1);
}

__global__ void __launch_bounds__(kFinishThreads) k_finish_init(const double* part0,
                                                              const double* part1, double* sc,
                                                              int* flags) {
  const double rz = ordered_sum(part0), bb = ordered_sum(part1);
  if (threadIdx.x != 0) return;
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

__global__ void __launch_bounds__(kFinishThreads) k_finish_pq(const double* part0, double* sc,
                                                            int* flags) {
  if (flags[F_STATE] != ST_RUN) return;
  const double pq = ordered_sum(part0);
  if (threadIdx.x != 0) return;
  sc[S_PQ] = pq;
  if (!isfinite(pq))
    flags[F_STATE] = ST_NAN;
  else if (!(pq > 0.0))
    flags[F_STATE] = ST_BREAK;
  else
    sc[S_ALPHA] = sc[S_RZ] / pq;
}

// p.q from the apply's per-block partials (count of them), summed in a fixed order: thread t
// adds part[t], part[t + 1024], ... in order, then the block tree.
__global__ void __launch_bounds__(kFinishThreads) k_finish_pq_var(const double* part,
                                                                int64_t count, double* sc,
                                                                int* flags) {
  if (flags[F_STATE] != ST_RUN) return;
  __shared__ double col[kFinishThreads];
  double v = 0.0;
  for (int64_t i = threadIdx.x; i < count; i += kFinishThreads) v += part[i];
  col[threadIdx.x] = v;
  __syncthreads();
  const double pq = ordered_sum(col);
  if (threadIdx.x != 0) return;
  sc[S_PQ] = pq;
  if (!isfinite(pq))
    flags[F_STATE] = ST_NAN;
  else if (!(pq > 0.0))
    flags[F_STATE] = ST_BREAK;
  else
    sc[S_ALPHA] = sc[S_RZ] / pq;
}

// x += alpha p, r -= alpha (1-m) q, z = D^-1 r; the r.z and r.r partials, accumulated in FP64.

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
    const double zi = d ? ri * d[i] : (bnd ? 0.0 : ri);
    z[i] = zi;
    s_rz = fma(ri, zi, s_rz);
    s_rr = fma(ri, ri, s_rr);
  }
  block_sum2(s_rz, s_rr, part0, part1);
}

__global__ void __launch_bounds__(kFinishThreads) k_finish_update(const double* part0,
                                                                const double* part1, double* sc,
                                                                int* flags, double rtol,
                                                                int maxit) {
  if (flags[F_STATE] != ST_RUN) return;
  const double rz = ordered_sum(part0), rr = ordered_sum(part1);
  if (threadIdx.x != 0) return;
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

// p = z + beta p, and q = 0 for the next apply's atomic scatter-add.
__global__ void __launch_bounds__(kReduceThreads) k_pupdate(double* __restrict__ p,
                                                            const double* __restrict__ z,
                                                            double* __restrict__ q, int64_t n,
                                                            const double* sc, const int* flags) {
  if (flags[F_STATE] != ST_RUN) return;
  const double beta = sc[S_BETA];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    p[i] = fma(beta, p[i], z[i]);
    q[i] = 0.0;
  }
}

// Jacobi: the diagonal is replaced in place by its inverse, 0 on the boundary (so z = dinv r is
// masked for free and the iteration needs no FP64 division -- slow on GB300's FP64 pipe); any
// non-positive interior entry is reported through flags as a breakdown.
__global__ void __launch_bounds__(kReduceThreads) k_fix_diag(double* __restrict__ d,
                                                             const uint8_t* __restrict__ mask,
                                                             int64_t n, int* flags) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (mask[i]) {
      d[i] = 0.0;
    } else {
      const double di = d[i];
      if (!(di > 0.0)) atomicExch(&flags[2], 1);
      d[i] = 1.0 / di;
    }
  }
}

// ||(1-m)(b - q)||^2 partials for the true residual; the residual itself is stored in rout
// when given.
__global__ void __launch_bounds__(kReduceThreads) k_resid(const double* __restrict__ b,
                                                          const double* __restrict__ q,
                                                          const uint8_t* __restrict__ mask,
                                                          double* __restrict__ rout, int64_t n,
                                                          double* part0, double* part1) {
  double s = 0.0, sb = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const bool bnd = mask[i] != 0;
    const double bi = bnd ? 0.0 : b[i];
    const double ri = bnd ? 0.0 : bi - q[i];
    if (rout) rout[i] = ri;
    s = fma(ri, ri, s);
    sb = fma(bi, bi, sb);
  }
  block_sum2(s, sb, part0, part1);
}

// ---- Chebyshev polynomial preconditioner z = q(D^-1 A_bc) D^-1 r: k steps of the Chebyshev
// semi-iteration for D^-1 A z = D^-1 r from z = 0 on an interval [lo, hi] that contains the
// spectrum, so that 1 - lam q(lam) = T_k((theta - lam)/delta) / T_k(theta/delta) (theta, delta
// the interval's centre and half-width): positive q on (0, hi], a linear SPD preconditioner.
// Three-term recurrence in the directions d_j with host-computed coefficients; k - 1 applies.

// first step: d = dinv r / theta, z = d; the r.z partials when it is also the last step
__global__ void __launch_bounds__(kReduceThreads) k_cheb_first(const double* __restrict__ r,
                                                               const double* __restrict__ dinv,
                                                               double* __restrict__ dv,
                                                               double* __restrict__ z, int64_t n,
                                                               double inv_theta, double* part0,
                                                               const int* flags, int with_dot) {
  if (flags[F_STATE] != ST_RUN) return;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = r[i];
    const double di = dinv[i] * ri * inv_theta;
    dv[i] = di;
    z[i] = di;
    if (with_dot) acc = fma(ri, di, acc);
  }
  if (with_dot) block_sum2(acc, 0.0, part0, nullptr);
}

// step j: d = c1 d + c2 dinv (r - A z), z += d, and q2 (= A z, scatter target) zeroed for the
// next step's apply; the r.z partials on the last step
__global__ void __launch_bounds__(kReduceThreads) k_cheb_step(const double* __restrict__ r,
                                                              double* __restrict__ q2,
                                                              const double* __restrict__ dinv,
                                                              double* __restrict__ dv,
                                                              double* __restrict__ z, int64_t n,
                                                              double c1, double c2, double* part0,
                                                              const int* flags, int with_dot) {
  if (flags[F_STATE] != ST_RUN) return;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = r[i];
    const double di = fma(c1, dv[i], c2 * dinv[i] * (ri - q2[i]));
    dv[i] = di;
    const double zi = z[i] + di;
    z[i] = zi;
    q2[i] = 0.0;
    if (with_dot) acc = fma(ri, zi, acc);
  }
  if (with_dot) block_sum2(acc, 0.0, part0, nullptr);
}

// x += alpha p, r -= alpha (1-m) q; the r.r partials (into part1)
__global__ void __launch_bounds__(kReduceThreads) k_update_xr(double* __restrict__ x,
                                                              double* __restrict__ r,
                                                              const double* __restrict__ p,
                                                              const double* __restrict__ q,
                                                              const uint8_t* __restrict__ mask,
                                                              int64_t n, const double* sc,
                                                              double* part1, const int* flags) {
  if (flags[F_STATE] != ST_RUN) return;
  const double alpha = sc[S_ALPHA];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double qi = mask[i] ? 0.0 : q[i];
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, qi, r[i]);
    r[i] = ri;
    acc = fma(ri, ri, acc);
  }
  block_sum2(acc, 0.0, part1, nullptr);
}

// initial r.z of the Chebyshev-preconditioned start; beta = 0 so that k_pupdate sets p = z
__global__ void __launch_bounds__(kFinishThreads) k_finish_rz(const double* part0, double* sc,
                                                            int* flags) {
  if (flags[F_STATE] != ST_RUN) return;
  const double rz = ordered_sum(part0);
  if (threadIdx.x != 0) return;
  sc[S_RZ] = rz;
  sc[S_BETA] = 0.0;
  if (!isfinite(rz))
    flags[F_STATE] = ST_NAN;
  else if (!(rz > 0.0))
    flags[F_STATE] = ST_BREAK;
}

// power iteration for the largest eigenvalue of D^-1 A_bc: start vector (interior dofs, hashed
// signs and magnitudes in [0.5, 1)), v = dinv w, and the generalised Rayleigh quotient
// (v.Av) / (v.Dv) partials
__global__ void __launch_bounds__(kReduceThreads) k_power_init(double* __restrict__ v,
                                                               const uint8_t* __restrict__ mask,
                                                               int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t h = (uint64_t)i * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
    h ^= h >> 31;
    h *= 0xBF58476D1CE4E5B9ull;
    h ^= h >> 29;
    const double u = 0.5 + 0.5 * (double)(h >> 11) * (1.0 / 9007199254740992.0);
    v[i] = mask[i] ? 0.0 : ((h & 1) ? u : -u);
  }
}

__global__ void __launch_bounds__(kReduceThreads) k_power_scale(double* __restrict__ w,
                                                                const double* __restrict__ dinv,
                                                                double* __restrict__ v,
                                                                int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    v[i] = dinv[i] * w[i];
    w[i] = 0.0;
  }
}

__global__ void __launch_bounds__(kReduceThreads) k_power_rq(const double* __restrict__ v,
                                                             const double* __restrict__ w,
                                                             const double* __restrict__ dinv,
                                                             int64_t n, double* part0,
                                                             double* part1) {
  double num = 0.0, den = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double di = dinv[i];
    if (di > 0.0) {
      num = fma(v[i], w[i], num);
      den = fma(v[i], v[i] / di, den);
    }
  }
  block_sum2(num, den, part0, part1);
}

__global__ void __launch_bounds__(kFinishThreads) k_finish2(const double* part0,
                                                          const double* part1, double* sc) {
  const double a = ordered_sum(part0), b = ordered_sum(part1);
  if (threadIdx.x == 0) {
    sc[S_TRUE] = a;
    sc[S_BB] = b;
  }
}

// ||(1-m)(b - A x)|| / ||(1-m) b|| into sc[S_TRUE] (0 when b vanishes), ||(1-m) b||^2 into sc[S_BB].
__global__ void __launch_bounds__(kFinishThreads) k_finish_resid(const double* part0,
                                                               const double* part1, double* sc) {
  const double rr = ordered_sum(part0), bb = ordered_sum(part1);
  if (threadIdx.x == 0) {
    sc[S_BB] = bb;
    sc[S_TRUE] = bb > 0.0 ? sqrt(rr / bb) : 0.0;
  }
}

}  // namespace

namespace {

// ---- FP32 inner solves of fe_pcg_ir: the same iteration on float vectors (FP32 pipe and half
//      the bytes; GB300's FP64 pipe makes even FP64 vector updates expensive).  Thread sums are
//      float, block partials double, so the reductions stay deterministic.

__global__ void __launch_bounds__(kReduceThreads) k_init32(const float* __restrict__ b,
                                                           const float* __restrict__ dinv,
                                                           float* __restrict__ x,
                                                           float* __restrict__ r,
                                                           float* __restrict__ z,
                                                           float* __restrict__ p,
                                                           float* __restrict__ q, int64_t n,
                                                           double* part0, double* part1) {
  float s_rz = 0.0f, s_bb = 0.0f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float bi = b[i];  // already masked
    const float zi = dinv ? bi * dinv[i] : bi;
    x[i] = 0.0f;
    r[i] = bi;
    z[i] = zi;
    p[i] = zi;
    q[i] = 0.0f;
    s_rz = fmaf(bi, zi, s_rz);
    s_bb = fmaf(bi, bi, s_bb);
  }
  block_sum2((double)s_rz, (double)s_bb, part0, part1);
}

__global__ void __launch_bounds__(kReduceThreads) k_update32(float* __restrict__ x,
                                                             float* __restrict__ r,
                                                             float* __restrict__ z,
                                                             const float* __restrict__ p,
                                                             const float* __restrict__ q,
                                                             const float* __restrict__ dinv,
                                                             const uint8_t* __restrict__ mask,
                                                             int64_t n, const double* sc,
                                                             double* part0, double* part1,
                                                             const int* flags) {
  if (flags[F_STATE] != ST_RUN) return;
  const float alpha = (float)sc[S_ALPHA];
  float s_rz = 0.0f, s_rr = 0.0f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const bool bnd = mask[i] != 0;
    const float qi = bnd ? 0.0f : q[i];
    x[i] = fmaf(alpha, p[i], x[i]);
    const float ri = fmaf(-alpha, qi, r[i]);
    r[i] = ri;
    const float zi = dinv ? ri * dinv[i] : (bnd ? 0.0f : ri);
    z[i] = zi;
    s_rz = fmaf(ri, zi, s_rz);
    s_rr = fmaf(ri, ri, s_rr);
  }
  block_sum2((double)s_rz, (double)s_rr, part0, part1);
}

__global__ void __launch_bounds__(kReduceThreads) k_pupdate32(float* __restrict__ p,
                                                              const float* __restrict__ z,
                                                              float* __restrict__ q, int64_t n,
                                                              const double* sc, const int* flags) {
  if (flags[F_STATE] != ST_RUN) return;
  const float beta = (float)sc[S_BETA];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    p[i] = fmaf(beta, p[i], z[i]);
    q[i] = 0.0f;
  }
}

// dst = src * 2^sshift as float (the outer residual as the inner right-hand side), and the FP32
// inverse diagonal d64 * 2^dshift when given (power-of-two scales: exact before the rounding).
__global__ void __launch_bounds__(kReduceThreads) k_to32(const double* __restrict__ src,
                                                         float* __restrict__ dst, int sshift,
                                                         const double* __restrict__ d64,
                                                         float* __restrict__ d32, int dshift,
                                                         int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    dst[i] = __double2float_rn(ldexp(src[i], sshift));
    if (d32) d32[i] = __double2float_rn(ldexp(d64[i], dshift));
  }
}

// x += dx * 2^shift (exact widening and scaling by integer manipulation)
__global__ void __launch_bounds__(kReduceThreads) k_axpy32(double* __restrict__ x,
                                                           const float* __restrict__ dx,
                                                           int64_t n, int shift) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] += fe::f64_from_f32_scaled(dx[i], shift);
}

}  // namespace

namespace {

struct PcgWork {
  double *r, *z, *p, *q, *d;
  double *part0, *part1, *sc;
  int* flags;
};

struct PcgResult {
  int state = ST_RUN, iters = 0, launches = 0;
  double rel = 0.0, bb = 0.0;
};

// Carves the work vectors (nvec of ndofs) and the reduction area out of the handle's cached
// workspace, (re)allocating it when the mesh size or the vector count grows.
int pcg_workspace(fe_pa* pa, int nvec, PcgWork* w, double** extra) {
  const int64_t n = pa->mesh->ndofs;
  if (pa->work_ndofs != n * nvec) {
    cudaFree(pa->d_work);
    cudaFree(pa->d_red);
    cudaFree(pa->d_flags);
    pa->d_work = pa->d_red = nullptr;
    pa->d_flags = nullptr;
    pa->work_ndofs = 0;
    cudaError_t err;
    if ((err = cudaMalloc(&pa->d_work, sizeof(double) * nvec * n)) != cudaSuccess ||
        (err = cudaMalloc(&pa->d_red, sizeof(double) * (2 * kReduceBlocks + kScalars))) !=
            cudaSuccess ||
        (err = cudaMalloc(&pa->d_flags, sizeof(int) * 4)) != cudaSuccess)
      return cuda_error(err, "fe_pcg: workspace cudaMalloc");
    pa->work_ndofs = n * nvec;
  }
  w->r = pa->d_work;
  w->z = w->r + n;
  w->p = w->z + n;
  w->q = w->p + n;
  w->d = w->q + n;
  if (extra) *extra = w->d + n;
  w->part0 = pa->d_red;
  w->part1 = w->part0 + kReduceBlocks;
  w->sc = w->part1 + kReduceBlocks;
  w->flags = pa->d_flags;
  return FE_OK;
}

// Jacobi diagonal into w.d (boundary entries 1); FE_ERR_BREAKDOWN on a non-positive entry.
int pcg_jacobi(const fe_pa* pa, int op, const PcgWork& w, cudaStream_t s, int* launches) {
  cudaError_t err;
  if ((err = cudaMemsetAsync(w.flags, 0, sizeof(int) * 4, s)) != cudaSuccess)
    return cuda_error(err, "fe_pcg: flags");
  int st = fe_assemble_diagonal(pa, op, w.d, s);
  if (st != FE_OK) return st;
  k_fix_diag<<<kReduceBlocks, kReduceThreads, 0, s>>>(w.d, pa->mesh->d_mask, pa->mesh->ndofs, w.flags);
  if ((err = cudaGetLastError()) != cudaSuccess) return cuda_error(err, "fe_pcg: diag fix launch");
  *launches += 2;
  int hflags[4];
  if ((err = cudaMemcpyAsync(hflags, w.flags, sizeof(int) * 4, cudaMemcpyDeviceToHost, s)) !=
          cudaSuccess ||
      (err = cudaStreamSynchronize(s)) != cudaSuccess)
    return cuda_error(err, "fe_pcg: diagonal");
  if (hflags[2]) return set_error(FE_ERR_BREAKDOWN, "fe_pcg: non-positive diagonal entry");
  return FE_OK;
}

// The CG iteration proper: solves A_bc x = b from x = 0 with the given apply variant and the
// Jacobi diagonal dj (or none); synchronous; res gets the state, iterations and launches.
int pcg_run(fe_pa* pa, int op, int variant, const double* b, double* x, const double* dj,
            double rtol, int maxit, const PcgWork& w, cudaStream_t s, PcgResult* res) {
  const fe_mesh* m = pa->mesh;
  const int64_t n = m->ndofs;
  const uint8_t* mask = m->d_mask;
  cudaError_t err;
  // p.Ap fused into the apply (per-block partials) except for the DMMA kernel
  const bool fused_dot = (variant != FE_VARIANT_F64_DMMA);
  int64_t nblk = 0;
  if (fused_dot) {
    int st = apply_dispatch(pa, op, variant, nullptr, nullptr, s, nullptr, nullptr, &nblk, true);
    if (st != FE_OK) return st;
    if (nblk > pa->dpart_cap) {
      cudaFree(pa->d_dpart);
      pa->d_dpart = nullptr;
      pa->dpart_cap = 0;
      if ((err = cudaMalloc(&pa->d_dpart, sizeof(double) * nblk)) != cudaSuccess)
        return cuda_error(err, "fe_pcg: partials cudaMalloc");
      pa->dpart_cap = nblk;
    }
  }
  if ((err = cudaMemsetAsync(w.flags, 0, sizeof(int) * 4, s)) != cudaSuccess)
    return cuda_error(err, "fe_pcg: flags");
  k_init<<<kReduceBlocks, kReduceThreads, 0, s>>>(b, mask, dj, x, w.r, w.z, w.p, w.q, n, w.part0,
                                                  w.part1);
  k_finish_init<<<1, kFinishThreads, 0, s>>>(w.part0, w.part1, w.sc, w.flags);
  if ((err = cudaGetLastError()) != cudaSuccess) return cuda_error(err, "fe_pcg: init launch");
  res->launches += 2;
  // `count` iterations on stream q; returns the kernels enqueued through *nk
  auto enqueue = [&](cudaStream_t q, int count, int* nk) -> int {
    for (int j = 0; j < count; ++j) {
      if (fused_dot) {
        int st = apply_dispatch(pa, op, variant, w.p, w.q, q, w.flags, pa->d_dpart);
        if (st != FE_OK) return st;
        k_finish_pq_var<<<1, kFinishThreads, 0, q>>>(pa->d_dpart, nblk, w.sc, w.flags);
        *nk += 2;
      } else {
        int st = apply_dispatch(pa, op, variant, w.p, w.q, q, w.flags);
        if (st != FE_OK) return st;
        k_dot<<<kReduceBlocks, kReduceThreads, 0, q>>>(w.p, w.q, n, w.part0, w.flags);
        k_finish_pq<<<1, kFinishThreads, 0, q>>>(w.part0, w.sc, w.flags);
        *nk += 3;
      }
      k_update<<<kReduceBlocks, kReduceThreads, 0, q>>>(x, w.r, w.z, w.p, w.q, dj, mask, n, w.sc,
                                                          w.part0, w.part1, w.flags);
      k_finish_update<<<1, kFinishThreads, 0, q>>>(w.part0, w.part1, w.sc, w.flags, rtol, maxit);
      k_pupdate<<<kReduceBlocks, kReduceThreads, 0, q>>>(w.p, w.z, w.q, n, w.sc, w.flags);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_error(e, "fe_pcg: iteration launch");
      *nk += 3;
    }
    return FE_OK;
  };
  int hflags[4] = {0, 0, 0, 0};
  int queued = 0;
  GraphBatch graph;
  for (;;) {
    const int count = maxit - queued < kBatch ? maxit - queued : kBatch;
    if (queued > 0 && count == kBatch && pa->pcg_graphs && !graph.failed && !graph.exec) {
      // the first batch ran eagerly (first-use kernel attributes are set); capture the next
      int nk = 0;
      graph.capture([&](cudaStream_t q) { return enqueue(q, kBatch, &nk); });
      graph.kernels = nk;
    }
    if (graph.exec && count == kBatch) {
      if ((err = cudaGraphLaunch(graph.exec, s)) != cudaSuccess)
        return cuda_error(err, "fe_pcg: graph launch");
      res->launches += graph.kernels;
    } else {
      int st = enqueue(s, count, &res->launches);
      if (st != FE_OK) return st;
    }
    queued += count;
    if ((err = cudaMemcpyAsync(hflags, w.flags, sizeof(int) * 4, cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess ||
        (err = cudaStreamSynchronize(s)) != cudaSuccess)
      return cuda_error(err, "fe_pcg: iteration");
    if (hflags[F_STATE] != ST_RUN || queued >= maxit) break;
  }
  double hsc[kScalars];
  if ((err = cudaMemcpyAsync(hsc, w.sc, sizeof(double) * kScalars, cudaMemcpyDeviceToHost, s)) !=
          cudaSuccess ||
      (err = cudaStreamSynchronize(s)) != cudaSuccess)
    return cuda_error(err, "fe_pcg: stats");
  res->state = hflags[F_STATE];
  res->iters = hflags[F_ITERS];
  res->rel = hsc[S_REL];
  res->bb = hsc[S_BB];
  return FE_OK;
}

// ||(1-m)(b - A x)|| / ||b|| with the given variant (q is overwritten); also stores the
// residual in rout when given, and its norm in *rnorm when given.
int pcg_true_residual(const fe_pa* pa, int op, int variant, const double* b, const double* x,
                      double* rout, const PcgWork& w, cudaStream_t s, int* launches,
                      double* rel, double* rnorm = nullptr) {
  const int64_t n = pa->mesh->ndofs;
  int st = apply_dispatch(pa, op, variant, x, w.q, s);
  if (st != FE_OK) return st;
  k_resid<<<kReduceBlocks, kReduceThreads, 0, s>>>(b, w.q, pa->mesh->d_mask, rout, n, w.part0,
                                                   w.part1);
  k_finish_resid<<<1, kFinishThreads, 0, s>>>(w.part0, w.part1, w.sc);
  cudaError_t err;
  if ((err = cudaGetLastError()) != cudaSuccess) return cuda_error(err, "fe_pcg: residual launch");
  *launches += 3;
  double hsc[kScalars];
  if ((err = cudaMemcpyAsync(hsc, w.sc, sizeof(double) * kScalars, cudaMemcpyDeviceToHost, s)) !=
          cudaSuccess ||
      (err = cudaStreamSynchronize(s)) != cudaSuccess)
    return cuda_error(err, "fe_pcg: residual");
  *rel = hsc[S_TRUE];
  if (rnorm) *rnorm = hsc[S_TRUE] * std::sqrt(hsc[S_BB]);
  return FE_OK;
}

// Inner solve of fe_pcg_ir on FP32 vectors: A_bc x = b from x = 0 with the FP32 apply.
struct PcgWork32 {
  float *r, *z, *p, *q, *dinv, *x;
};

int pcg_run_f32(fe_pa* pa, int op, const float* b, const PcgWork32& v, bool jacobi, double rtol,
                int maxit, const PcgWork& w, cudaStream_t s, PcgResult* res) {
  const fe_mesh* m = pa->mesh;
  const int64_t n = m->ndofs;
  cudaError_t err;
  int64_t nblk = 0;
  int st = apply_dispatch(pa, op, FE_VARIANT_F32, nullptr, nullptr, s, nullptr, nullptr, &nblk, true);
  if (st != FE_OK) return st;
  if (nblk > pa->dpart_cap) {
    cudaFree(pa->d_dpart);
    pa->d_dpart = nullptr;
    pa->dpart_cap = 0;
    if ((err = cudaMalloc(&pa->d_dpart, sizeof(double) * nblk)) != cudaSuccess)
      return cuda_error(err, "fe_pcg_ir: partials cudaMalloc");
    pa->dpart_cap = nblk;
  }
  const float* dinv = jacobi ? v.dinv : nullptr;
  if ((err = cudaMemsetAsync(w.flags, 0, sizeof(int) * 4, s)) != cudaSuccess)
    return cuda_error(err, "fe_pcg_ir: flags");
  k_init32<<<kReduceBlocks, kReduceThreads, 0, s>>>(b, dinv, v.x, v.r, v.z, v.p, v.q, n, w.part0,
                                                    w.part1);
  k_finish_init<<<1, kFinishThreads, 0, s>>>(w.part0, w.part1, w.sc, w.flags);
  if ((err = cudaGetLastError()) != cudaSuccess) return cuda_error(err, "fe_pcg_ir: init launch");
  res->launches += 2;
  int hflags[4] = {0, 0, 0, 0};
  int queued = 0;
  for (;;) {
    for (int j = 0; j < kBatch && queued < maxit; ++j, ++queued) {
      st = apply_f32_vectors(pa, op, v.p, v.q, s, w.flags, pa->d_dpart);
      if (st != FE_OK) return st;
      k_finish_pq_var<<<1, kFinishThreads, 0, s>>>(pa->d_dpart, nblk, w.sc, w.flags);
      k_update32<<<kReduceBlocks, kReduceThreads, 0, s>>>(v.x, v.r, v.z, v.p, v.q, dinv, m->d_mask,
                                                          n, w.sc, w.part0, w.part1, w.flags);
      k_finish_update<<<1, kFinishThreads, 0, s>>>(w.part0, w.part1, w.sc, w.flags, rtol, maxit);
      k_pupdate32<<<kReduceBlocks, kReduceThreads, 0, s>>>(v.p, v.z, v.q, n, w.sc, w.flags);
      if ((err = cudaGetLastError()) != cudaSuccess)
        return cuda_error(err, "fe_pcg_ir: iteration launch");
      res->launches += 5;
    }
    if ((err = cudaMemcpyAsync(hflags, w.flags, sizeof(int) * 4, cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess ||
        (err = cudaStreamSynchronize(s)) != cudaSuccess)
      return cuda_error(err, "fe_pcg_ir: iteration");
    if (hflags[F_STATE] != ST_RUN || queued >= maxit) break;
  }
  res->state = hflags[F_STATE];
  res->iters = hflags[F_ITERS];
  return FE_OK;
}

// Largest eigenvalue estimate of D^-1 A_bc: `iters` power steps from a fixed pseudo-random
// start, then the generalised Rayleigh quotient (v.Av)/(v.Dv) of the last iterate (a lower
// bound that converges from below).  dinv: inverse diagonal, 0 on the boundary.  v, w: work.
int cheb_lmax(const fe_pa* pa, int op, int variant, const double* dinv, double* v, double* w,
              const PcgWork& ws, cudaStream_t s, int iters, int* launches, double* out) {
  const int64_t n = pa->mesh->ndofs;
  cudaError_t err;
  k_power_init<<<kReduceBlocks, kReduceThreads, 0, s>>>(v, pa->mesh->d_mask, n);
  ++*launches;
  for (int it = 0; it < iters; ++it) {
    int st = apply_dispatch(pa, op, variant, v, w, s);
    if (st != FE_OK) return st;
    k_power_scale<<<kReduceBlocks, kReduceThreads, 0, s>>>(w, dinv, v, n);
    *launches += 2;
  }
  int st = apply_dispatch(pa, op, variant, v, w, s);
  if (st != FE_OK) return st;
  k_power_rq<<<kReduceBlocks, kReduceThreads, 0, s>>>(v, w, dinv, n, ws.part0, ws.part1);
  k_finish2<<<1, kFinishThreads, 0, s>>>(ws.part0, ws.part1, ws.sc);
  *launches += 3;
  double hsc[kScalars];
  if ((err = cudaGetLastError()) != cudaSuccess ||
      (err = cudaMemcpyAsync(hsc, ws.sc, sizeof(double) * kScalars, cudaMemcpyDeviceToHost, s)) !=
          cudaSuccess ||
      (err = cudaStreamSynchronize(s)) != cudaSuccess)
    return cuda_error(err, "fe_pcg_chebyshev: eigenvalue estimate");
  const double lam = hsc[S_BB] > 0.0 ? hsc[S_TRUE] / hsc[S_BB] : 0.0;
  if (!(lam > 0.0) || !std::isfinite(lam))
    return set_error(FE_ERR_BREAKDOWN, "fe_pcg_chebyshev: no positive eigenvalue estimate");
  *out = lam;
  return FE_OK;
}

// PCG with the Chebyshev preconditioner of `degree` steps on [lo, hi]; same conventions as
// pcg_run (x = 0 start, device-resident state, batches of kBatch iterations between flag
// reads).  dv, q2: two extra work vectors.
int pcg_run_cheb(fe_pa* pa, int op, int variant, const double* b, double* x, const double* dinv,
                 int degree, double lo, double hi, double rtol, int maxit, const PcgWork& w,
                 double* dv, double* q2, cudaStream_t s, PcgResult* res) {
  const fe_mesh* m = pa->mesh;
  const int64_t n = m->ndofs;
  const uint8_t* mask = m->d_mask;
  cudaError_t err;
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo);
  std::vector<double> c1(degree, 0.0), c2(degree, 0.0);
  double rho = delta / theta;
  for (int j = 1; j < degree; ++j) {
    const double rn = 1.0 / (2.0 * theta / delta - rho);
    c1[j] = rn * rho;
    c2[j] = 2.0 * rn / delta;
    rho = rn;
  }
  const bool fused_dot = (variant != FE_VARIANT_F64_DMMA);
  int64_t nblk = 0;
  if (fused_dot) {
    int st = apply_dispatch(pa, op, variant, nullptr, nullptr, s, nullptr, nullptr, &nblk, true);
    if (st != FE_OK) return st;
    if (nblk > pa->dpart_cap) {
      cudaFree(pa->d_dpart);
      pa->d_dpart = nullptr;
      pa->dpart_cap = 0;
      if ((err = cudaMalloc(&pa->d_dpart, sizeof(double) * nblk)) != cudaSuccess)
        return cuda_error(err, "fe_pcg_chebyshev: partials cudaMalloc");
      pa->dpart_cap = nblk;
    }
  }
  // z = q(D^-1 A) D^-1 r into w.z, the r.z partials into w.part0 (skipped once stopped)
  auto precondition = [&]() -> int {
    k_cheb_first<<<kReduceBlocks, kReduceThreads, 0, s>>>(w.r, dinv, dv, w.z, n, 1.0 / theta,
                                                          w.part0, w.flags, degree == 1);
    ++res->launches;
    for (int j = 1; j < degree; ++j) {
      int st = apply_dispatch(pa, op, variant, w.z, q2, s, w.flags);
      if (st != FE_OK) return st;
      k_cheb_step<<<kReduceBlocks, kReduceThreads, 0, s>>>(w.r, q2, dinv, dv, w.z, n, c1[j], c2[j],
                                                           w.part0, w.flags, j == degree - 1);
      res->launches += 2;
    }
    return FE_OK;
  };
  if ((err = cudaMemsetAsync(w.flags, 0, sizeof(int) * 4, s)) != cudaSuccess ||
      (err = cudaMemsetAsync(q2, 0, sizeof(double) * n, s)) != cudaSuccess)
    return cuda_error(err, "fe_pcg_chebyshev: init");
  k_init<<<kReduceBlocks, kReduceThreads, 0, s>>>(b, mask, dinv, x, w.r, w.z, w.p, w.q, n, w.part0,
                                                  w.part1);
  k_finish_init<<<1, kFinishThreads, 0, s>>>(w.part0, w.part1, w.sc, w.flags);
  res->launches += 2;
  int st = precondition();
  if (st != FE_OK) return st;
  k_finish_rz<<<1, kFinishThreads, 0, s>>>(w.part0, w.sc, w.flags);
  k_pupdate<<<kReduceBlocks, kReduceThreads, 0, s>>>(w.p, w.z, w.q, n, w.sc, w.flags);
  if ((err = cudaGetLastError()) != cudaSuccess) return cuda_error(err, "fe_pcg_chebyshev: start");
  res->launches += 2;
  int hflags[4] = {0, 0, 0, 0};
  int queued = 0;
  for (;;) {
    for (int j = 0; j < kBatch && queued < maxit; ++j, ++queued) {
      if (fused_dot) {
        if ((st = apply_dispatch(pa, op, variant, w.p, w.q, s, w.flags, pa->d_dpart)) != FE_OK)
          return st;
        k_finish_pq_var<<<1, kFinishThreads, 0, s>>>(pa->d_dpart, nblk, w.sc, w.flags);
        res->launches += 2;
      } else {
        if ((st = apply_dispatch(pa, op, variant, w.p, w.q, s, w.flags)) != FE_OK) return st;
        k_dot<<<kReduceBlocks, kReduceThreads, 0, s>>>(w.p, w.q, n, w.part0, w.flags);
        k_finish_pq<<<1, kFinishThreads, 0, s>>>(w.part0, w.sc, w.flags);
        res->launches += 3;
      }
      k_update_xr<<<kReduceBlocks, kReduceThreads, 0, s>>>(x, w.r, w.p, w.q, mask, n, w.sc,
                                                           w.part1, w.flags);
      ++res->launches;
      if ((st = precondition()) != FE_OK) return st;
      k_finish_update<<<1, kFinishThreads, 0, s>>>(w.part0, w.part1, w.sc, w.flags, rtol, maxit);
      k_pupdate<<<kReduceBlocks, kReduceThreads, 0, s>>>(w.p, w.z, w.q, n, w.sc, w.flags);
      if ((err = cudaGetLastError()) != cudaSuccess)
        return cuda_error(err, "fe_pcg_chebyshev: iteration launch");
      res->launches += 2;
    }
    if ((err = cudaMemcpyAsync(hflags, w.flags, sizeof(int) * 4, cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess ||
        (err = cudaStreamSynchronize(s)) != cudaSuccess)
      return cuda_error(err, "fe_pcg_chebyshev: iteration");
    if (hflags[F_STATE] != ST_RUN || queued >= maxit) break;
  }
  double hsc[kScalars];
  if ((err = cudaMemcpyAsync(hsc, w.sc, sizeof(double) * kScalars, cudaMemcpyDeviceToHost, s)) !=
          cudaSuccess ||
      (err = cudaStreamSynchronize(s)) != cudaSuccess)
    return cuda_error(err, "fe_pcg_chebyshev: stats");
  res->state = hflags[F_STATE];
  res->iters = hflags[F_ITERS];
  res->rel = hsc[S_REL];
  res->bb = hsc[S_BB];
  return FE_OK;
}

int pcg_status(int state, const char* who) {
  switch (state) {
    case ST_CONV:
      return FE_OK;
    case ST_BREAK:
      return set_error(FE_ERR_BREAKDOWN, std::string(who) + ": p.Ap <= 0 (operator not SPD on the free dofs)");
    case ST_NAN:
      return set_error(FE_ERR_NAN, std::string(who) + ": NaN or Inf in the iteration");
    default:
      return set_error(FE_ERR_NOT_CONVERGED, std::string(who) + ": maxit reached before rtol");
  }
}

int pcg_check_args(const fe_pa* pa, int op, int pc, const double* b, const double* x, double rtol,
                   int maxit, const char* who) {
  if (!pa || !b || !x) return set_error(FE_ERR_ARG, std::string(who) + ": null argument");
  if (op != FE_DIFFUSION && op != FE_MASS) return set_error(FE_ERR_ARG, std::string(who) + ": bad op");
  if (!(pa->ops & op)) return set_error(FE_ERR_ARG, std::string(who) + ": operator not set up");
  if (pc != FE_PC_NONE && pc != FE_PC_JACOBI)
    return set_error(FE_ERR_ARG, std::string(who) + ": bad preconditioner");
  if (maxit < 1 || !(rtol >= 0.0)) return set_error(FE_ERR_ARG, std::string(who) + ": bad rtol or maxit");
  return FE_OK;
}

// Solvers that iterate with the handle's variant need an FP64-accurate one.
int pcg_check_variant(const fe_pa* pa, const char* who) {
  if (pa->variant == FE_VARIANT_F32)
    return set_error(FE_ERR_UNSUPPORTED, std::string(who) + ": the FP32 variant is not "
                                         "FP64-accurate; select FE_VARIANT_F64, F32X2 or "
                                         "F64_DMMA (or use fe_pcg_ir)");
  return FE_OK;
}


}  // namespace

extern "C" int fe_pcg(fe_pa* pa, int op, int pc, const double* dev_b, double* dev_x, double rtol,
                      int maxit, fe_pcg_stats* stats, void* stream) {
  clear_error();
  if (pc == FE_PC_CHEBYSHEV)
    return fe_pcg_chebyshev(pa, op, 0, 0.0, 0.0, dev_b, dev_x, rtol, maxit, stats, stream);
  if (pc == FE_PC_LEARNED) {
    if (!pa) return set_error(FE_ERR_ARG, "fe_pcg: pa is NULL");
    if (!pa->lpc)
      return set_error(FE_ERR_ARG, "fe_pcg: FE_PC_LEARNED needs fe_pa_set_learned first");
    return fe_fcg(pa, op, pa->lpc, dev_b, dev_x, rtol, maxit, stats, stream);
  }
  const auto t0 = std::chrono::steady_clock::now();
  if (stats) *stats = fe_pcg_stats{0, 0.0, 0.0, 0.0, 0, 0};
  int st = pcg_check_args(pa, op, pc, dev_b, dev_x, rtol, maxit, "fe_pcg");
  if (st == FE_OK) st = pcg_check_variant(pa, "fe_pcg");
  if (st != FE_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  PcgWork w;
  if ((st = pcg_workspace(pa, 5, &w, nullptr)) != FE_OK) return st;
  PcgResult res;
  if (pc == FE_PC_JACOBI && (st = pcg_jacobi(pa, op, w, s, &res.launches)) != FE_OK) return st;
  st = pcg_run(pa, op, pa->variant, dev_b, dev_x, pc == FE_PC_JACOBI ? w.d : nullptr, rtol, maxit,
               w, s, &res);
  if (st != FE_OK) return st;
  double true_rel = 0.0;  // with the FP64 operator whatever the iteration's variant
  if ((st = pcg_true_residual(pa, op, FE_VARIANT_F64, dev_b, dev_x, nullptr, w, s, &res.launches,
                              &true_rel)) != FE_OK)
    return st;
  if (stats) {
    stats->iters = res.iters;
    stats->rel_resid = res.rel;
    stats->true_rel_resid = true_rel;
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    stats->launches = res.launches;
    stats->outer_iters = 1;
  }
  return pcg_status(res.state, "fe_pcg");
}

extern "C" int fe_pcg_host(fe_pa* pa, int op, int pc, const double* host_b, double* host_x,
                           double rtol, int maxit, fe_pcg_stats* stats, void* stream) {
  clear_error();
  const auto t0 = std::chrono::steady_clock::now();
  if (stats) *stats = fe_pcg_stats{0, 0.0, 0.0, 0.0, 0, 0};
  if (!pa || !pa->mesh) return set_error(FE_ERR_ARG, "fe_pcg_host: pa is NULL");
  if (!host_b || !host_x) return set_error(FE_ERR_ARG, "fe_pcg_host: host_b or host_x is NULL");
  const int64_t n = pa->mesh->ndofs;
  cudaError_t err;
  if (!pa->d_hostio) {
    if ((err = cudaMalloc(&pa->d_hostio, sizeof(double) * 2 * n)) != cudaSuccess) {
      pa->d_hostio = nullptr;
      return cuda_error(err, "fe_pcg_host: device b and x");
    }
  }
  double* db = pa->d_hostio;
  double* dx = pa->d_hostio + n;
  cudaStream_t s = (cudaStream_t)stream;
  if ((err = cudaMemcpyAsync(db, host_b, sizeof(double) * n, cudaMemcpyHostToDevice, s)) !=
      cudaSuccess)
    return cuda_error(err, "fe_pcg_host: copy b to the device");
  const int st = fe_pcg(pa, op, pc, db, dx, rtol, maxit, stats, stream);
  if (st != FE_OK && st != FE_ERR_NOT_CONVERGED && st != FE_ERR_BREAKDOWN && st != FE_ERR_NAN) {
    cudaStreamSynchronize(s);  // the copy of host_b has ended when the call returns
    return st;
  }
  if ((err = cudaMemcpyAsync(host_x, dx, sizeof(double) * n, cudaMemcpyDeviceToHost, s)) !=
      cudaSuccess)
    return cuda_error(err, "fe_pcg_host: copy x to the host");
  if ((err = cudaStreamSynchronize(s)) != cudaSuccess)
    return cuda_error(err, "fe_pcg_host: synchronize");
  if (stats)
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return st;
}

extern "C" int fe_pcg_ir(fe_pa* pa, int op, int pc, const double* dev_b, double* dev_x,
                         double rtol, int maxit, double inner_rtol, fe_pcg_stats* stats,
                         void* stream) {
  clear_error();
  const auto t0 = std::chrono::steady_clock::now();
  if (stats) *stats = fe_pcg_stats{0, 0.0, 0.0, 0.0, 0, 0};
  int st = pcg_check_args(pa, op, pc, dev_b, dev_x, rtol, maxit, "fe_pcg_ir");
  if (st != FE_OK) return st;
  if (inner_rtol == 0.0) inner_rtol = 1e-2;
  if (!(inner_rtol > 0.0 && inner_rtol < 1.0))
    return set_error(FE_ERR_ARG, "fe_pcg_ir: inner_rtol must lie in (0, 1)");
  cudaStream_t s = (cudaStream_t)stream;
  // The outer residual is FP64 (FP64 data and arithmetic).  The inner solves run on
  // A32 = 2^-qs A (the FP32 data carry the shift qs that puts them in the float range) with
  // the right-hand side r 2^-e (e the exponent of ||r||, so that it stays in the float range as
  // the refinement shrinks r); their solution d32 = A32^-1 r 2^-e gives d = 2^(e - qs) d32.
  const int hi = FE_VARIANT_F64;
  if ((op == FE_DIFFUSION ? pa->d_qd_diff32 : pa->d_qd_mass32) == nullptr) {
    const int saved = pa->variant;
    if ((st = fe_pa_set_variant(pa, FE_VARIANT_F32, stream)) != FE_OK) return st;
    pa->variant = saved;
  }
  PcgWork w;
  double* extra = nullptr;
  // 5 FP64 work vectors + the FP64 outer residual + 7 FP32 vectors (4 doubles' worth)
  if ((st = pcg_workspace(pa, 10, &w, &extra)) != FE_OK) return st;
  const int64_t n = pa->mesh->ndofs;
  double* rr = extra;                        // outer residual (FP64)
  float* f32base = reinterpret_cast<float*>(extra + n);
  PcgWork32 v{f32base, f32base + n, f32base + 2 * n, f32base + 3 * n, f32base + 4 * n,
              f32base + 5 * n};
  float* b32 = f32base + 6 * n;  // inner right-hand side
  PcgResult res;
  if (pc == FE_PC_JACOBI && (st = pcg_jacobi(pa, op, w, s, &res.launches)) != FE_OK) return st;
  cudaError_t err;
  if ((err = cudaMemsetAsync(dev_x, 0, sizeof(double) * n, s)) != cudaSuccess)
    return cuda_error(err, "fe_pcg_ir: zero x");
  const int qs = pa->qd32_shift[op == FE_DIFFUSION ? 0 : 1];
  double rel = 1.0, rnorm = 0.0;
  if ((st = pcg_true_residual(pa, op, hi, dev_b, dev_x, rr, w, s, &res.launches, &rel, &rnorm)) !=
      FE_OK)
    return st;
  int outer = 0, inner_total = 0, state = (rel <= rtol) ? ST_CONV : ST_RUN;
  bool dinv_ready = false;
  while (state == ST_RUN) {
    if (!std::isfinite(rel)) {
      state = ST_NAN;
      break;
    }
    // inner FP32 solve of A32 d32 = r 2^-e to inner_rtol relative to its right-hand side
    int e = 0;
    std::frexp(rnorm, &e);
    k_to32<<<kReduceBlocks, kReduceThreads, 0, s>>>(
        rr, b32, -e, w.d, (pc == FE_PC_JACOBI && !dinv_ready) ? v.dinv : nullptr, qs, n);
    dinv_ready = true;
    res.launches += 1;
    PcgResult in;
    st = pcg_run_f32(pa, op, b32, v, pc == FE_PC_JACOBI, inner_rtol, maxit - inner_total, w, s,
                     &in);
    if (st != FE_OK) return st;
    res.launches += in.launches;
    inner_total += in.iters;
    ++outer;
    if (in.state == ST_NAN) {
      state = ST_NAN;
      break;
    }
    if (in.state == ST_BREAK) {
      state = ST_BREAK;
      break;
    }
    k_axpy32<<<kReduceBlocks, kReduceThreads, 0, s>>>(dev_x, v.x, n, e - qs);
    if ((err = cudaGetLastError()) != cudaSuccess) return cuda_error(err, "fe_pcg_ir: update launch");
    res.launches += 1;
    const double prev = rel;
    if ((st = pcg_true_residual(pa, op, hi, dev_b, dev_x, rr, w, s, &res.launches, &rel,
                                &rnorm)) != FE_OK)
      return st;
    if (rel <= rtol)
      state = ST_CONV;
    else if (inner_total >= maxit || !(rel < prev))
      state = ST_MAXIT;  // budget spent, or refinement stagnated at the inner precision
  }
  if (stats) {
    stats->iters = inner_total;
    stats->rel_resid = rel;
    stats->true_rel_resid = rel;
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    stats->launches = res.launches;
    stats->outer_iters = outer;
  }
  return pcg_status(state, "fe_pcg_ir");
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
  if (stats) *stats = fe_pcg_stats{0, 0.0, 0.0, 0.0, 0, 0};
  int launches = 0;
  if (!pa || !dev_b || !dev_x) return set_error(FE_ERR_ARG, "fe_pcg_noalloc: null argument");
  if (op != FE_DIFFUSION && op != FE_MASS) return set_error(FE_ERR_ARG, "fe_pcg_noalloc: bad op");
  if (!(pa->ops & op)) return set_error(FE_ERR_ARG, "fe_pcg_noalloc: operator not set up");
  if (pc != FE_PC_NONE && pc != FE_PC_JACOBI)
    return set_error(FE_ERR_ARG, "fe_pcg_noalloc: bad preconditioner");
  if (maxit < 1 || !(rtol >= 0.0)) return set_error(FE_ERR_ARG, "fe_pcg_noalloc: bad rtol or maxit");
  int st = pcg_check_variant(pa, "fe_pcg_noalloc");
  if (st != FE_OK) return st;
  const fe_mesh* m = pa->mesh;
  const int64_t n = m->ndofs;
  if (n > kNoAllocMaxDofs)
    return set_error(FE_ERR_ARG, "fe_pcg_noalloc: the mesh has " + std::to_string(n) +
                                     " dofs, more than the fixed scratch holds (" +
                                     std::to_string(kNoAllocMaxDofs) + "); use fe_pcg");
  double* base = nullptr;
  st = noalloc_scratch(&base);
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
  // and partial is written before it is read (d by the diagonal assembly, q by k_init and
  // k_pupdate)
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
  k_init<<<kReduceBlocks, kReduceThreads, 0, s>>>(dev_b, mask, dj, dev_x, r, z, p, q, n, part0,
                                                   part1);
  k_finish_init<<<1, kFinishThreads, 0, s>>>(part0, part1, sc, flags);
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
      st = apply_dispatch(pa, op, pa->variant, p, q, s, flags);
      if (st != FE_OK) return st;
      k_dot<<<kReduceBlocks, kReduceThreads, 0, s>>>(p, q, n, part0, flags);
      k_finish_pq<<<1, kFinishThreads, 0, s>>>(part0, sc, flags);
      k_update<<<kReduceBlocks, kReduceThreads, 0, s>>>(dev_x, r, z, p, q, dj, mask, n, sc, part0,
                                                          part1, flags);
      k_finish_update<<<1, kFinishThreads, 0, s>>>(part0, part1, sc, flags, rtol, maxit);
      k_pupdate<<<kReduceBlocks, kReduceThreads, 0, s>>>(p, z, q, n, sc, flags);
      NOALLOC_LAUNCH_CHECK("fe_pcg_noalloc: iteration launch");
      launches += 6;
    }
    if ((err = cudaMemcpyAsync(hflags, flags, sizeof(int) * 4, cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess ||
        (err = cudaStreamSynchronize(s)) != cudaSuccess)
      return cuda_error(err, "fe_pcg_noalloc: iteration");
    if (hflags[F_STATE] != ST_RUN || queued >= maxit) break;
  }
  st = apply_dispatch(pa, op, FE_VARIANT_F64, dev_x, q, s);  // FP64 true residual
  if (st != FE_OK) return st;
  k_resid<<<kReduceBlocks, kReduceThreads, 0, s>>>(dev_b, q, mask, nullptr, n, part0, part1);
  k_finish_resid<<<1, kFinishThreads, 0, s>>>(part0, part1, sc);
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
    stats->outer_iters = 1;
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

namespace {
constexpr int kChebDegree = 4;       // default steps of the Chebyshev preconditioner
constexpr double kChebRatio = 30.0;  // default hi / lo of its interval
constexpr double kChebSafety = 1.1;  // hi = kChebSafety x the power-iteration estimate
constexpr int kPowerIters = 20;
}  // namespace

extern "C" int fe_estimate_lmax(fe_pa* pa, int op, int iters, double* lmax, void* stream) {
  clear_error();
  if (!pa || !lmax) return set_error(FE_ERR_ARG, "fe_estimate_lmax: null argument");
  if (op != FE_DIFFUSION && op != FE_MASS) return set_error(FE_ERR_ARG, "fe_estimate_lmax: bad op");
  if (!(pa->ops & op)) return set_error(FE_ERR_ARG, "fe_estimate_lmax: operator not set up");
  if (iters < 0 || iters > 1000) return set_error(FE_ERR_ARG, "fe_estimate_lmax: iters in 0..1000");
  cudaStream_t s = (cudaStream_t)stream;
  PcgWork w;
  double* extra = nullptr;
  int st;
  if ((st = pcg_workspace(pa, 7, &w, &extra)) != FE_OK) return st;
  int launches = 0;
  if ((st = pcg_jacobi(pa, op, w, s, &launches)) != FE_OK) return st;
  const int64_t n = pa->mesh->ndofs;
  return cheb_lmax(pa, op, pa->variant, w.d, extra, extra + n, w, s, iters, &launches, lmax);
}

extern "C" int fe_pcg_chebyshev(fe_pa* pa, int op, int degree, double lmax, double lmin_ratio,
                                const double* dev_b, double* dev_x, double rtol, int maxit,
                                fe_pcg_stats* stats, void* stream) {
  clear_error();
  const auto t0 = std::chrono::steady_clock::now();
  if (stats) *stats = fe_pcg_stats{0, 0.0, 0.0, 0.0, 0, 0};
  int st = pcg_check_args(pa, op, FE_PC_JACOBI, dev_b, dev_x, rtol, maxit, "fe_pcg_chebyshev");
  if (st == FE_OK) st = pcg_check_variant(pa, "fe_pcg_chebyshev");
  if (st != FE_OK) return st;
  if (degree == 0) degree = kChebDegree;
  if (lmin_ratio == 0.0) lmin_ratio = kChebRatio;
  if (degree < 1 || degree > 32)
    return set_error(FE_ERR_ARG, "fe_pcg_chebyshev: degree must lie in 1..32");
  if (!(lmin_ratio > 1.0) || !(lmax >= 0.0) || !std::isfinite(lmax))
    return set_error(FE_ERR_ARG, "fe_pcg_chebyshev: need lmin_ratio > 1 and lmax >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  PcgWork w;
  double* extra = nullptr;
  if ((st = pcg_workspace(pa, 7, &w, &extra)) != FE_OK) return st;
  const int64_t n = pa->mesh->ndofs;
  PcgResult res;
  if ((st = pcg_jacobi(pa, op, w, s, &res.launches)) != FE_OK) return st;
  double hi = lmax;
  if (hi == 0.0) {
    double& cached = pa->cheb_lmax[op == FE_DIFFUSION ? 0 : 1];
    if (cached <= 0.0 &&
        (st = cheb_lmax(pa, op, pa->variant, w.d, extra, extra + n, w, s, kPowerIters,
                        &res.launches, &cached)) != FE_OK)
      return st;
    hi = kChebSafety * cached;
  }
  if ((st = pcg_run_cheb(pa, op, pa->variant, dev_b, dev_x, w.d, degree, hi / lmin_ratio, hi, rtol,
                         maxit, w, extra, extra + n, s, &res)) != FE_OK)
    return st;
  double true_rel = 0.0;  // with the FP64 operator whatever the iteration's variant
  if ((st = pcg_true_residual(pa, op, FE_VARIANT_F64, dev_b, dev_x, nullptr, w, s, &res.launches,
                              &true_rel)) != FE_OK)
    return st;
  if (stats) {
    stats->iters = res.iters;
    stats->rel_resid = res.rel;
    stats->true_rel_resid = true_rel;
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    stats->launches = res.launches;
    stats->outer_iters = 1;
  }
  return pcg_status(res.state, "fe_pcg_chebyshev");
}

extern "C" int fe_pcg_set_graphs(fe_pa* pa, int enable) {
  clear_error();
  if (!pa) return set_error(FE_ERR_ARG, "fe_pcg_set_graphs: pa is NULL");
  pa->pcg_graphs = enable != 0;
  return FE_OK;
}
