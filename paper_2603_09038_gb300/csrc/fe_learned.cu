// Learned element-patch preconditioner and flexible CG (an extension; the paper has no learned
// component).
//
// Preconditioner:  z = sum_e R_e^T W_e S_e s_e f(x_e / s_e),  x_e = S_e W_e R_e r,  s_e = ||x_e||_2,
// with W_e = diag(1/multiplicity)^(1/2) on the element's dofs (0 on the Dirichlet boundary),
// S = diag(A)^(-1/2), and f(x) = relu(relu(x W1) W2) W3 + x W0: a bias-free three-layer MLP
// D^3 -> width -> width -> D^3 with ReLU plus a linear skip term, BF16 weights and activations,
// FP32 accumulation on the tensor cores; width 0 keeps only the linear map x W0.  With f(x) = S_e^{-1} A_ee^{-1} S_e^{-1} x exactly this is
// the symmetrically weighted additive Schwarz method on element patches, which needs about half
// the iterations of Jacobi on these problems (the one-sided weighting R^T W^2 A_ee^{-1} R does
// not beat Jacobi).  The symmetric diagonal scaling makes the map nearly the same on every
// element even across coefficient jumps, so one network serves the whole mesh.
//
// Training pairs come from the FP64-accurate operator itself: for interior elements, taken in
// classes of elements three apart in every direction (within a class no two neighbourhoods
// overlap), the block A_ee of the assembled matrix on the element's dofs is probed with D^3
// applies of the global operator per class,
// factored (batched FP64 Cholesky) and used to produce pairs x = S_e v, t = S_e^{-1} A_ee^{-1} v
// for v i.i.d. normal, v = A_ee u, and v = W_e r for residual snapshots r of Jacobi-FCG runs,
// both scaled by 1/||t||.
// Training minimises the relative squared error with Adam, all on the GPU with the kernels
// below.  The flexible CG (Notay's FCG(1)) tolerates the nonlinear preconditioner and falls back
// to Jacobi-PCG on its residual when it stagnates; convergence is judged on the FP64 residual.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <chrono>
#include <functional>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "fe_f2.h"
#include "fe_internal.h"
#include "fe_mlp.cuh"
#include "fe_mlp_tc.cuh"

using namespace fe;

namespace fe {
int lpc_apply(fe_lpc* L, const double* r, double* z, cudaStream_t s, bool accumulate = false);
}

struct fe_lpc {
  fe_pa* pa = nullptr;  // not owned
  int op = FE_DIFFUSION;
  int fallback = FE_PC_JACOBI;  // what fe_fcg continues with once the network is given up
  int din = 0, width = 0;
  int64_t nparam = 0;
  float* w32 = nullptr;         // packed FP32 master weights W1 | W2 | W3
  __nv_bfloat16* wb = nullptr;  // BF16 copy used by the GEMMs
  float *adam_m = nullptr, *adam_v = nullptr, *grad = nullptr;
  int adam_t = 0;
  double* wsq = nullptr;        // (1/multiplicity)^(1/2) per dof, 0 on the boundary
  double* dinv = nullptr;       // inverse diagonal, 0 on the boundary (Jacobi)
  double* dis = nullptr;        // diagonal^(-1/2), 0 on the boundary
  double* fsc = nullptr;        // wsq * dis: the input/output scaling F = W S of the apply
  float* fsc32 = nullptr;       // the same in FP32 (read by the fused kernel)
  __nv_bfloat16* wimg = nullptr;  // shared-memory weight image of the fused apply
  bool wimg_ok = false;
  int fused_grid = 0;           // persistent grid of the fused apply (0: unfused GEMM path)
  __nv_bfloat16* tcimg = nullptr;  // canonical K-major weight images of the tcgen05 apply
  bool tcimg_ok = false;
  int tc_grid = 0;              // persistent grid of the tcgen05 apply (0: not built / no fit)
  int tc_grid32 = 0;            // the same for FP32 vectors
  int* d_tcfail = nullptr;      // raised by the tcgen05 apply when it gives up a wait
  int kernel = FE_LPC_KERNEL_AUTO;  // which inference kernel fe_lpc_apply and the solvers use
  // training samples
  int64_t nsamp = 0;
  __nv_bfloat16* Xs = nullptr;  // [nsamp][din]
  float* Ts = nullptr;          // [nsamp][din]
  uint64_t seed = 0;
  // forward/backward workspace for up to cap rows
  int64_t cap = 0;
  __nv_bfloat16 *Xb = nullptr, *H1b = nullptr, *H2b = nullptr, *dYb = nullptr, *dA1b = nullptr,
                *dA2b = nullptr;
  float *Z1 = nullptr, *Z2 = nullptr, *Y = nullptr, *Tb = nullptr, *scale = nullptr;
  double* red = nullptr;        // loss reductions
};

namespace {

constexpr int kT = 256;
constexpr int kLpcMaxOrder = 8;          // Cholesky of A_ee: whole block or panels in smem
constexpr int64_t kProbeDoubles = 1 << 28;  // bound on the probed blocks (2 GB)

__device__ __forceinline__ uint64_t mix64(uint64_t z) {  // splitmix64 finaliser
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double normal01(uint64_t key) {  // Box-Muller on two hashed uniforms
  const uint64_t a = mix64(key), b = mix64(key ^ 0xD1B54A32D192ED03ull);
  const double u1 = ((a >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  const double u2 = ((b >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

__global__ void k_init_weights(float* w, int din, int width, uint64_t seed) {
  const int64_t n1 = (int64_t)din * width, n2 = (int64_t)width * width, n3 = n1;
  const int64_t n = n1 + n2 + n3 + (int64_t)din * din;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int fan_in = i < n1 ? din : width;
    w[i] = i < n1 + n2 + n3
               ? (float)(normal01(seed * 0x100000001ull + (uint64_t)i) * sqrt(2.0 / fan_in))
               : 0.0f;  // skip term starts at zero
  }
}

__global__ void k_normal_vec(double* __restrict__ v, int64_t n, uint64_t seed) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] = normal01(seed + 0x9E3779B97F4A7C15ull * (uint64_t)i);
}

__global__ void k_to_bf16(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = __float2bfloat16(a[i]);
}

// multiplicity of every dof (elements sharing it), then wsq = mult^(-1/2) off the boundary
__global__ void k_count(const int32_t* __restrict__ map, int64_t n, double* __restrict__ c) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&c[map[i]], 1.0);
}

__global__ void k_wsq(double* __restrict__ c, const uint8_t* __restrict__ mask, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    c[i] = mask[i] ? 0.0 : 1.0 / sqrt(c[i]);
}

__global__ void k_invert_diag(double* __restrict__ d, const uint8_t* __restrict__ mask, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    d[i] = (mask[i] || !(d[i] > 0.0)) ? 0.0 : 1.0 / d[i];
}

// b = sqrt(a) and c = w * b
__global__ void k_sqrt_vec(const double* __restrict__ a, double* __restrict__ b,
                           const double* __restrict__ w, double* __restrict__ c, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double bi = sqrt(a[i]);
    b[i] = bi;
    c[i] = w[i] * bi;
  }
}

// ---- probing of A_ee for the sample elements
__global__ void k_probe_set(double* __restrict__ v, const int32_t* __restrict__ map,
                            const int32_t* __restrict__ elems, int ns, int din, int a) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < ns) v[map[(int64_t)elems[s] * din + a]] = 1.0;
}

__global__ void k_probe_get(const double* __restrict__ w, const int32_t* __restrict__ map,
                            const int32_t* __restrict__ elems, int ns, int din, int a,
                            double* __restrict__ Aee) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)ns * din) return;
  const int s = (int)(i / din), b = (int)(i % din);
  Aee[((int64_t)s * din + b) * din + a] = w[map[(int64_t)elems[s] * din + b]];
}

// Batched Cholesky A = L L^T in place (lower triangle), one block per matrix; FP64.
__global__ void k_cholesky(double* __restrict__ Aee, int din, int* __restrict__ fail) {
  extern __shared__ double sm[];
  double* A = Aee + (int64_t)blockIdx.x * din * din;
  for (int i = threadIdx.x; i < din * din; i += blockDim.x) sm[i] = A[i];
  __syncthreads();
  for (int k = 0; k < din; ++k) {
    if (threadIdx.x == 0) {
      const double d = sm[k * din + k];
      if (!(d > 0.0)) atomicExch(fail, 1);
      sm[k * din + k] = sqrt(d > 0.0 ? d : 1.0);
    }
    __syncthreads();
    const double lkk = sm[k * din + k];
    for (int i = k + 1 + threadIdx.x; i < din; i += blockDim.x) sm[i * din + k] /= lkk;
    __syncthreads();
    for (int idx = threadIdx.x; idx < (din - k - 1) * (din - k - 1); idx += blockDim.x) {
      const int i = k + 1 + idx / (din - k - 1), j = k + 1 + idx % (din - k - 1);
      if (j <= i) sm[i * din + j] -= sm[i * din + k] * sm[j * din + k];
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < din * din; i += blockDim.x) A[i] = sm[i];
}

// Batched Cholesky for blocks too large for one block's shared memory (D^3 > 125): one thread
// block per matrix, right-looking by panels of kPanel columns.  Each panel (its rows kb..n-1) is
// loaded into shared memory, factored there column by column, written back, and then applied
// to the trailing lower triangle (A[i][j] -= sum_c L[i][c] L[j][c]) with both factors read from
// shared memory, so the trailing matrix in global memory is read and written once per panel.
constexpr int kPanel = 32;

__global__ void __launch_bounds__(256) k_cholesky_blocked(double* __restrict__ Aee, int din,
                                                          int* __restrict__ fail) {
  extern __shared__ double pn[];  // [din][kPanel]: rows kb.. of the current panel
  double* A = Aee + (int64_t)blockIdx.x * din * din;
  for (int kb = 0; kb < din; kb += kPanel) {
    const int w = din - kb < kPanel ? din - kb : kPanel;
    const int rows = din - kb;
    for (int t = threadIdx.x; t < rows * w; t += blockDim.x) {
      const int i = t / w, c = t - i * w;
      pn[i * kPanel + c] = A[(int64_t)(kb + i) * din + kb + c];
    }
    __syncthreads();
    for (int c = 0; c < w; ++c) {
      if (threadIdx.x == 0) {
        const double d = pn[c * kPanel + c];
        if (!(d > 0.0)) atomicExch(fail, 1);
        pn[c * kPanel + c] = sqrt(d > 0.0 ? d : 1.0);
      }
      __syncthreads();
      const double lcc = pn[c * kPanel + c];
      for (int i = c + 1 + threadIdx.x; i < rows; i += blockDim.x) pn[i * kPanel + c] /= lcc;
      __syncthreads();
      // the rest of the panel: columns c' in (c, w), rows i >= c'
      const int nc = w - c - 1;
      for (int t = threadIdx.x; t < (rows - c - 1) * nc; t += blockDim.x) {
        const int i = c + 1 + t / nc, cp = c + 1 + t % nc;
        if (i >= cp) pn[i * kPanel + cp] -= pn[i * kPanel + c] * pn[cp * kPanel + c];
      }
      __syncthreads();
    }
    for (int t = threadIdx.x; t < rows * w; t += blockDim.x) {
      const int i = t / w, c = t - i * w;
      if (i >= c) A[(int64_t)(kb + i) * din + kb + c] = pn[i * kPanel + c];
    }
    // trailing update of the lower triangle: rows and columns kb + w .. din - 1
    const int m = rows - w;
    const int64_t ntri = (int64_t)m * (m + 1) / 2;
    for (int64_t t = threadIdx.x; t < ntri; t += blockDim.x) {
      // (i, j) with 0 <= j <= i < m from the triangular index t = i (i + 1) / 2 + j
      int i = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
      while ((int64_t)i * (i + 1) / 2 > t) --i;
      while ((int64_t)(i + 1) * (i + 2) / 2 <= t) ++i;
      const int j = (int)(t - (int64_t)i * (i + 1) / 2);
      const double* li = pn + (w + i) * kPanel;
      const double* lj = pn + (w + j) * kPanel;
      double acc = 0.0;
      for (int c = 0; c < w; ++c) acc = fma(li[c], lj[c], acc);
      A[(int64_t)(kb + w + i) * din + kb + w + j] -= acc;
    }
    __syncthreads();
  }
}

// Samples: per sample element s and replica q, v is (q mod 3) i.i.d. normal, A_ee u for normal u
// (then A_ee^{-1} v = u), or W_e r for a residual snapshot r of a Jacobi-FCG run; u = A_ee^{-1} v
// by the Cholesky factors; x = S v and t = u / S, both stored scaled by 1/||t||.
__global__ void k_samples(const double* __restrict__ Lfac, const double* __restrict__ snaps,
                          int nsnap,
                          const int32_t* __restrict__ map, const int32_t* __restrict__ elems,
                          const double* __restrict__ dis, const double* __restrict__ wsq,
                          int ns, int din, int reps,
                          uint64_t seed, __nv_bfloat16* __restrict__ Xs, float* __restrict__ Ts,
                          double* __restrict__ Xd, double* __restrict__ Td) {
  extern __shared__ double sh[];
  double* r = sh;
  double* t = sh + din;
  double* u = sh + 2 * din;
  const int s = blockIdx.x;
  const double* L = Lfac + (int64_t)s * din * din;
  for (int q = 0; q < reps; ++q) {
    const int64_t row = (int64_t)s * reps + q;
    const int kind = q % 3;
    const bool applied = kind == 1;
    const double* snap = snaps + ((int64_t)((q / 3) % nsnap) * ns + s) * din;
    for (int i = threadIdx.x; i < din; i += blockDim.x)
      u[i] = kind == 2 ? snap[i] * wsq[map[(int64_t)elems[s] * din + i]]
                       : normal01(seed ^ ((uint64_t)row * 1315423911ull + (uint64_t)i * 2654435761ull));
    __syncthreads();
    if (threadIdx.x == 0) {
      if (applied) {  // r = A_ee u = L (L^T u)
        for (int i = 0; i < din; ++i) {
          double acc = 0.0;
          for (int j = i; j < din; ++j) acc += L[(int64_t)j * din + i] * u[j];
          t[i] = acc;
        }
        for (int i = din - 1; i >= 0; --i) {
          double acc = 0.0;
          for (int j = 0; j <= i; ++j) acc += L[(int64_t)i * din + j] * t[j];
          r[i] = acc;
        }
        for (int i = 0; i < din; ++i) t[i] = u[i];
      } else {
        for (int i = 0; i < din; ++i) r[i] = u[i];
        for (int i = 0; i < din; ++i) {  // L y = r
          double acc = r[i];
          for (int j = 0; j < i; ++j) acc -= L[(int64_t)i * din + j] * t[j];
          t[i] = acc / L[(int64_t)i * din + i];
        }
        for (int i = din - 1; i >= 0; --i) {  // L^T t = y
          double acc = t[i];
          for (int j = i + 1; j < din; ++j) acc -= L[(int64_t)j * din + i] * t[j];
          t[i] = acc / L[(int64_t)i * din + i];
        }
      }
      double nt = 0.0;
      for (int i = 0; i < din; ++i) {
        const double si = dis[map[(int64_t)elems[s] * din + i]];  // > 0 on interior elements
        u[i] = si * r[i];
        t[i] /= si;
        nt += t[i] * t[i];
      }
      // Pairs are scaled to ||t|| = 1, so that the batch loss is the mean relative error per
      // sample: with 1/||x|| the smooth modes (large t for a small x) would dominate it and the
      // high-frequency response, where a poor preconditioner hurts most, would go unfitted.  The
      // network is positively homogeneous, so the scale of a pair changes only its weight.
      nt = sqrt(nt);
      const double inv = nt > 0.0 ? 1.0 / nt : 0.0;
      for (int i = 0; i < din; ++i) {
        Xs[row * din + i] = __float2bfloat16((float)(u[i] * inv));
        Ts[row * din + i] = (float)(t[i] * inv);
      }
      if (Xd) {  // FP64 copies before the rounding (test hook)
        for (int i = 0; i < din; ++i) {
          Xd[row * din + i] = u[i] * inv;
          Td[row * din + i] = t[i] * inv;
        }
      }
    }
    __syncthreads();
  }
}

// batch rows gathered from the sample set by a hashed index per (step, row)
__global__ void k_batch(const __nv_bfloat16* __restrict__ Xs, const float* __restrict__ Ts,
                        int64_t nsamp, int din, int batch, uint64_t key,
                        __nv_bfloat16* __restrict__ Xb, float* __restrict__ Tb) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)batch * din) return;
  const int b = (int)(i / din), c = (int)(i % din);
  const int64_t src = (int64_t)(mix64(key + (uint64_t)b) % (uint64_t)nsamp);
  Xb[i] = Xs[src * din + c];
  Tb[i] = Ts[src * din + c];
}

// sum (y - t)^2 and sum t^2 (atomics into red[0], red[1])
__global__ void k_loss_terms(const float* __restrict__ Y, const float* __restrict__ T, int64_t n,
                             double* __restrict__ red) {
  double a = 0.0, b = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double d = (double)Y[i] - (double)T[i];
    a += d * d;
    b += (double)T[i] * (double)T[i];
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&red[0], a);
    atomicAdd(&red[1], b);
  }
}

__global__ void k_dY(const float* __restrict__ Y, const float* __restrict__ T, int64_t n,
                     const double* __restrict__ red, __nv_bfloat16* __restrict__ dY) {
  const float sc = (float)(2.0 / red[1]);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dY[i] = __float2bfloat16(sc * (Y[i] - T[i]));
}

__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps,
                       float c1, float c2, __nv_bfloat16* __restrict__ wb) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    wb[i] = __float2bfloat16(wi);
  }
}

// preconditioner input rows: x_e = F r on the element (F = W S), scaled to unit norm
__global__ void k_lpc_gather(const double* __restrict__ r, const int32_t* __restrict__ map,
                             const double* __restrict__ fsc,
                             int64_t e0, int64_t nrows, int din, __nv_bfloat16* __restrict__ X,
                             float* __restrict__ scale) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  if (row >= nrows) return;
  const int32_t* m = map + (e0 + row) * din;
  double ss = 0.0;
  for (int a = lane; a < din; a += 32) {
    const double xi = fsc[m[a]] * r[m[a]];
    ss += xi * xi;
  }
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  const double s = sqrt(ss);
  const double inv = s > 0.0 ? 1.0 / s : 0.0;
  for (int a = lane; a < din; a += 32)
    X[row * din + a] = __float2bfloat16((float)(fsc[m[a]] * r[m[a]] * inv));
  if (lane == 0) scale[row] = (float)s;
}

__global__ void k_lpc_scatter(const float* __restrict__ Y, const float* __restrict__ scale,
                              const int32_t* __restrict__ map, const double* __restrict__ fsc,
                              int64_t e0, int64_t nrows, int din, double* __restrict__ z) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrows * din) return;
  const int64_t row = i / din;
  const int32_t g = map[(e0 + row) * din + (i % din)];
  const double w = fsc[g];
  if (w != 0.0) atomicAdd(&z[g], w * (double)scale[row] * (double)Y[i]);
}

unsigned int grid1(int64_t n) {
  int64_t g = (n + kT - 1) / kT;
  if (g > 152 * 32) g = 152 * 32;
  return (unsigned int)(g < 1 ? 1 : g);
}

int ensure_workspace(fe_lpc* L, int64_t rows) {
  if (rows <= L->cap) return FE_OK;
  cudaFree(L->Xb); cudaFree(L->H1b); cudaFree(L->H2b); cudaFree(L->dYb); cudaFree(L->dA1b);
  cudaFree(L->dA2b); cudaFree(L->Z1); cudaFree(L->Z2); cudaFree(L->Y); cudaFree(L->Tb);
  cudaFree(L->scale);
  L->cap = 0;
  // hidden-layer buffers get at least 16 bytes so that width 0 (no hidden layers) allocates too
  const int64_t w = L->width > 0 ? L->width : 1, d = L->din;
  cudaError_t err;
  if ((err = cudaMalloc(&L->Xb, 2 * rows * d)) != cudaSuccess ||
      (err = cudaMalloc(&L->H1b, 2 * rows * w)) != cudaSuccess ||
      (err = cudaMalloc(&L->H2b, 2 * rows * w)) != cudaSuccess ||
      (err = cudaMalloc(&L->dYb, 2 * rows * d)) != cudaSuccess ||
      (err = cudaMalloc(&L->dA1b, 2 * rows * w)) != cudaSuccess ||
      (err = cudaMalloc(&L->dA2b, 2 * rows * w)) != cudaSuccess ||
      (err = cudaMalloc(&L->Z1, 4 * rows * w)) != cudaSuccess ||
      (err = cudaMalloc(&L->Z2, 4 * rows * w)) != cudaSuccess ||
      (err = cudaMalloc(&L->Y, 4 * rows * d)) != cudaSuccess ||
      (err = cudaMalloc(&L->Tb, 4 * rows * d)) != cudaSuccess ||
      (err = cudaMalloc(&L->scale, 4 * rows)) != cudaSuccess)
    return cuda_error(err, "fe_lpc: workspace cudaMalloc");
  L->cap = rows;
  return FE_OK;
}

// Y = f(X) for `rows` rows already in L->Xb; the pre-activations Z1, Z2 are kept for the
// backward pass only when keep is set.
int mlp_forward(fe_lpc* L, int64_t rows, cudaStream_t s, bool keep = true) {
  const int d = L->din, w = L->width;
  if (w == 0) {  // the linear patch map: Y = X W0
    const cudaError_t e = mlp::gemm<false, false, mlp::EPI_STORE>((int)rows, d, d, L->Xb, d, L->wb,
                                                                   d, L->Y, d, nullptr, 0, s);
    return cuda_error(e, "fe_lpc: forward launch");
  }
  const __nv_bfloat16* W1 = L->wb;
  const __nv_bfloat16* W2 = W1 + (int64_t)d * w;
  const __nv_bfloat16* W3 = W2 + (int64_t)w * w;
  const __nv_bfloat16* W0 = W3 + (int64_t)w * d;
  cudaError_t err;
  if ((err = mlp::gemm<false, false, mlp::EPI_RELU_BF16>((int)rows, w, d, L->Xb, d, W1, w, keep ? L->Z1 : nullptr, w,
                                                         L->H1b, w, s)) != cudaSuccess ||
      (err = mlp::gemm<false, false, mlp::EPI_RELU_BF16>((int)rows, w, w, L->H1b, w, W2, w, keep ? L->Z2 : nullptr, w,
                                                         L->H2b, w, s)) != cudaSuccess ||
      (err = mlp::gemm<false, false, mlp::EPI_STORE>((int)rows, d, w, L->H2b, w, W3, d, L->Y, d,
                                                     nullptr, 0, s)) != cudaSuccess ||
      (err = mlp::gemm<false, false, mlp::EPI_ACCUM>((int)rows, d, d, L->Xb, d, W0, d, L->Y, d,
                                                     nullptr, 0, s)) != cudaSuccess)
    return cuda_error(err, "fe_lpc: forward launch");
  return FE_OK;
}

// loss and gradient (into L->grad) of the batch in L->Xb / L->Tb
int mlp_loss_grad(fe_lpc* L, int64_t rows, cudaStream_t s, double* loss_out) {
  int st = mlp_forward(L, rows, s);
  if (st != FE_OK) return st;
  const int d = L->din, w = L->width;
  const __nv_bfloat16* W2 = L->wb + (int64_t)d * w;
  const __nv_bfloat16* W3 = W2 + (int64_t)w * w;
  float* g1 = L->grad;
  float* g2 = g1 + (int64_t)d * w;
  float* g3 = g2 + (int64_t)w * w;
  float* g0 = g3 + (int64_t)w * d;
  cudaError_t err;
  if ((err = cudaMemsetAsync(L->red, 0, 2 * sizeof(double), s)) != cudaSuccess)
    return cuda_error(err, "fe_lpc: reduction");
  k_loss_terms<<<grid1(rows * d), kT, 0, s>>>(L->Y, L->Tb, rows * d, L->red);
  k_dY<<<grid1(rows * d), kT, 0, s>>>(L->Y, L->Tb, rows * d, L->red, L->dYb);
  if (w == 0) {  // linear map: dW0 = X^T dY
    if ((err = cudaGetLastError()) != cudaSuccess ||
        (err = mlp::gemm<true, false, mlp::EPI_STORE>(d, d, (int)rows, L->Xb, d, L->dYb, d, g0, d,
                                                      nullptr, 0, s)) != cudaSuccess)
      return cuda_error(err, "fe_lpc: backward launch");
  } else if ((err = cudaGetLastError()) != cudaSuccess ||
      (err = mlp::gemm<true, false, mlp::EPI_STORE>(w, d, (int)rows, L->H2b, w, L->dYb, d, g3, d,
                                                    nullptr, 0, s)) != cudaSuccess ||
      (err = mlp::gemm<false, true, mlp::EPI_RELU_MASK_BF16>((int)rows, w, d, L->dYb, d, W3, d,
                                                             L->Z2, w, L->dA2b, w, s)) != cudaSuccess ||
      (err = mlp::gemm<true, false, mlp::EPI_STORE>(w, w, (int)rows, L->H1b, w, L->dA2b, w, g2, w,
                                                    nullptr, 0, s)) != cudaSuccess ||
      (err = mlp::gemm<false, true, mlp::EPI_RELU_MASK_BF16>((int)rows, w, w, L->dA2b, w, W2, w,
                                                             L->Z1, w, L->dA1b, w, s)) != cudaSuccess ||
      (err = mlp::gemm<true, false, mlp::EPI_STORE>(d, w, (int)rows, L->Xb, d, L->dA1b, w, g1, w,
                                                    nullptr, 0, s)) != cudaSuccess ||
      (err = mlp::gemm<true, false, mlp::EPI_STORE>(d, d, (int)rows, L->Xb, d, L->dYb, d, g0, d,
                                                    nullptr, 0, s)) != cudaSuccess)
    return cuda_error(err, "fe_lpc: backward launch");
  if (loss_out) {
    double h[2];
    if ((err = cudaMemcpyAsync(h, L->red, 2 * sizeof(double), cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess ||
        (err = cudaStreamSynchronize(s)) != cudaSuccess)
      return cuda_error(err, "fe_lpc: loss");
    *loss_out = h[1] > 0.0 ? h[0] / h[1] : 0.0;
  }
  return FE_OK;
}

// ---- flexible CG
constexpr int kRB = 1024;  // reduction blocks (of kT threads); partials reduced by one block
constexpr int kStall = 500;  // learned preconditioner: iterations without a 1% gain before Jacobi

enum { S_PQ = 0, S_PR, S_RR, S_ZQ, S_ZR, S_BB, S_ALPHA, S_BETA, S_TRUE, S_N };

__device__ __forceinline__ void block_partial2(double a, double b, double* pa, double* pb) {
  __shared__ double sa[kT / 32], sb[kT / 32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x / 32;
  if ((threadIdx.x & 31) == 0) {
    sa[w] = a;
    sb[w] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0.0, tb = 0.0;
    for (int i = 0; i < kT / 32; ++i) {
      ta += sa[i];
      tb += sb[i];
    }
    pa[blockIdx.x] = ta;
    pb[blockIdx.x] = tb;
  }
}

// fixed-order sum of kRB partials by one block of kRB threads
__device__ __forceinline__ double finish_sum(const double* part) {
  __shared__ double sh[kRB];
  sh[threadIdx.x] = part[threadIdx.x];
  __syncthreads();
  for (int h = kRB / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
    __syncthreads();
  }
  const double t = sh[0];
  __syncthreads();
  return t;
}

// The FCG vector kernels take VT = double (the FP64 solver) or float (the inner solve of the
// mixed-precision refinement); thread-local sums are kept in VT -- float sums keep the float
// kernels off GB300's narrow FP64 pipe -- and only the block partials are FP64.

// r = (1-m) b, x = 0; partial ||r||^2
template <class VT>
__global__ void __launch_bounds__(kT) k_fcg_init(const VT* __restrict__ b,
                                                 const uint8_t* __restrict__ mask,
                                                 VT* __restrict__ x, VT* __restrict__ r,
                                                 int64_t n, double* part0, double* part1) {
  VT a = VT(0);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const VT ri = mask[i] ? VT(0) : b[i];
    r[i] = ri;
    x[i] = VT(0);
    a = fma(ri, ri, a);
  }
  block_partial2((double)a, 0.0, part0, part1);
}

// q masked on the boundary; partials p.q and p.r
template <class VT>
__global__ void __launch_bounds__(kT) k_fcg_pq(const VT* __restrict__ p, VT* __restrict__ q,
                                               const VT* __restrict__ r,
                                               const uint8_t* __restrict__ mask, int64_t n,
                                               double* part0, double* part1) {
  VT a = VT(0), c = VT(0);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    VT qi = q[i];
    if (mask[i]) {
      qi = VT(0);
      q[i] = VT(0);
    }
    a = fma(p[i], qi, a);
    c = fma(p[i], r[i], c);
  }
  block_partial2((double)a, (double)c, part0, part1);
}

// x += alpha p, r -= alpha q; partial ||r||^2
template <class VT>
__global__ void __launch_bounds__(kT) k_fcg_xr(VT* __restrict__ x, VT* __restrict__ r,
                                               const VT* __restrict__ p,
                                               const VT* __restrict__ q, int64_t n,
                                               const double* sc, double* part0, double* part1) {
  const VT alpha = (VT)sc[S_ALPHA];
  VT a = VT(0);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    x[i] = fma(alpha, p[i], x[i]);
    const VT ri = fma(-alpha, q[i], r[i]);
    r[i] = ri;
    a = fma(ri, ri, a);
  }
  block_partial2((double)a, 0.0, part0, part1);
}

// partials z.q and z.r
template <class VT>
__global__ void __launch_bounds__(kT) k_fcg_zq(const VT* __restrict__ z, const VT* __restrict__ q,
                                               const VT* __restrict__ r, int64_t n,
                                               double* part0, double* part1) {
  VT a = VT(0), c = VT(0);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    a = fma(z[i], q[i], a);
    c = fma(z[i], r[i], c);
  }
  block_partial2((double)a, (double)c, part0, part1);
}

// which: 0 init (bb, rr), 1 after p.q (alpha), 2 after the update (rr), 3 after z.q (beta)
__global__ void __launch_bounds__(kRB) k_fcg_finish(const double* part0, const double* part1,
                                                    double* sc, int which) {
  const double a = finish_sum(part0), b = finish_sum(part1);
  if (threadIdx.x != 0) return;
  if (which == 0) {
    sc[S_BB] = a;
    sc[S_RR] = a;
  } else if (which == 1) {
    sc[S_PQ] = a;
    sc[S_PR] = b;
    sc[S_ALPHA] = a != 0.0 ? b / a : 0.0;
  } else if (which == 2) {
    sc[S_RR] = a;
  } else if (which == 3) {
    sc[S_ZQ] = a;
    sc[S_ZR] = b;
    sc[S_BETA] = sc[S_PQ] != 0.0 ? -a / sc[S_PQ] : 0.0;
  } else {
    sc[S_TRUE] = a;
    sc[S_BB] = b;
  }
}

// z = dinv r (Jacobi; dinv is 0 on the boundary)
template <class VT>
__global__ void __launch_bounds__(kT) k_fcg_jacobi(const VT* __restrict__ dinv,
                                                   const VT* __restrict__ r, VT* __restrict__ z,
                                                   int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    z[i] = dinv[i] * r[i];
}

// p = z + beta p (beta from sc, or 0 for a restart); q = 0 for the next float apply
template <class VT>
__global__ void __launch_bounds__(kT) k_fcg_p(VT* __restrict__ p, const VT* __restrict__ z,
                                              VT* __restrict__ q, int64_t n, const double* sc,
                                              int restart) {
  const VT beta = restart ? VT(0) : (VT)sc[S_BETA];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    p[i] = fma(beta, p[i], z[i]);
    if (q) q[i] = VT(0);
  }
}

// partials ||(1-m)(b - q)||^2 and ||(1-m) b||^2
__global__ void __launch_bounds__(kT) k_fcg_resid(const double* __restrict__ b,
                                                  const double* __restrict__ q,
                                                  const uint8_t* __restrict__ mask, int64_t n,
                                                  double* part0, double* part1) {
  double a = 0.0, c = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (mask[i]) continue;
    const double d = b[i] - q[i];
    a = fma(d, d, a);
    c = fma(b[i], b[i], c);
  }
  block_partial2(a, c, part0, part1);
}

// r restricted to the sample elements -> out[s][a]
__global__ void k_snap(const double* __restrict__ r, const int32_t* __restrict__ map,
                       const int32_t* __restrict__ elems, int ns, int din,
                       double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)ns * din) return;
  out[i] = r[map[(int64_t)elems[i / din] * din + (i % din)]];
}

struct Snapshots {  // residual snapshots at the listed iterations (training data)
  const int32_t* elems = nullptr;
  int ns = 0, din = 0;
  std::vector<int> at;  // iterations, ascending
  double* out = nullptr;  // [at.size()][ns][din]
};

struct FcgResult {
  int iters = 0, launches = 0, restarts = 0, status = FE_OK;
  double rel = 0.0, true_rel = 0.0;
  bool stop_at_fallback = false;  // in: end the run where it would fall back to Jacobi
  bool handed_off = false;        // out: it did (x holds the iterate reached)
};

int lpc_apply32(fe_lpc* L, const float* r, float* z, cudaStream_t s);

// FCG from x = 0 on an n-vector system with boundary mask `mask`.  apply: out = A in (out
// overwritten); prec_learned: z = M(r) with the learned preconditioner, or empty for Jacobi
// throughout (z = dinv r); true_apply: the FP64 operator for the exit true residual (VT = double
// only).  snap_map: the element map the residual snapshots of the training data read through.
// Synchronous.  work: NULL, or 4 n VT values plus reduction space of 2 kRB + S_N doubles (red)
// supplied by the caller.
template <class VT>
int fcg_core(int64_t n, const uint8_t* mask, const int32_t* snap_map,
             const std::function<int(const VT*, VT*)>& apply,
             const std::function<int(const VT*, VT*)>& prec_learned,
             const std::function<int(const double*, double*)>& true_apply, const VT* dinv,
             const VT* b, VT* x, double rtol, int maxit, Snapshots* snap, cudaStream_t s,
             FcgResult* res, VT* work = nullptr, double* red_in = nullptr) {
  constexpr bool F64 = std::is_same<VT, double>::value;
  VT* vec = work;
  double* red = red_in;
  cudaError_t err;
  if (!vec && (err = cudaMalloc(&vec, sizeof(VT) * 4 * n)) != cudaSuccess)
    return cuda_error(err, "fe_fcg: workspace cudaMalloc");
  if (!red && (err = cudaMalloc(&red, sizeof(double) * (2 * kRB + S_N))) != cudaSuccess) {
    if (!work) cudaFree(vec);
    return cuda_error(err, "fe_fcg: workspace cudaMalloc");
  }
  VT *r = vec, *z = vec + n, *p = vec + 2 * n, *q = vec + 3 * n;
  double *part0 = red, *part1 = red + kRB, *sc = red + 2 * kRB;
  int st = FE_OK;
  bool learned = static_cast<bool>(prec_learned);
  size_t next_snap = 0;
  auto precond = [&]() -> int {
    res->launches += learned ? 2 : 1;
    if (learned) return prec_learned(r, z);
    k_fcg_jacobi<VT><<<kRB, kT, 0, s>>>(dinv, r, z, n);
    return FE_OK;
  };
  auto take_snap = [&](int it) {
    if constexpr (F64) {
      if (!snap) return;
      while (next_snap < snap->at.size() && snap->at[next_snap] == it) {
        k_snap<<<(unsigned int)(((int64_t)snap->ns * snap->din + kT - 1) / kT), kT, 0, s>>>(
            r, snap_map, snap->elems, snap->ns, snap->din,
            snap->out + (int64_t)next_snap * snap->ns * snap->din);
        ++next_snap;
      }
    }
  };
  double hsc[S_N];
  auto read_sc = [&]() -> int {
    cudaError_t e;
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(hsc, sc, sizeof(hsc), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
      return cuda_error(e, "fe_fcg: iteration");
    return FE_OK;
  };
  cudaMemsetAsync(sc, 0, sizeof(double) * S_N, s);
  k_fcg_init<VT><<<kRB, kT, 0, s>>>(b, mask, x, r, n, part0, part1);
  k_fcg_finish<<<1, kRB, 0, s>>>(part0, part1, sc, 0);
  res->launches += 2;
  take_snap(0);
  if ((st = precond()) == FE_OK) {
    k_fcg_zq<VT><<<kRB, kT, 0, s>>>(z, r, r, n, part0, part1);  // z.r (twice)
    k_fcg_finish<<<1, kRB, 0, s>>>(part0, part1, sc, 3);
    res->launches += 2;
    st = read_sc();
  }
  if (st == FE_OK && learned && hsc[S_BB] > 0.0 && !(hsc[S_ZR] > 0.0)) {
    learned = false;  // not a descent direction: Jacobi from the start
    ++res->restarts;
    if (res->stop_at_fallback)
      res->handed_off = true;
    else
      st = precond();
  }
  if (st == FE_OK) {
    k_fcg_p<VT><<<kRB, kT, 0, s>>>(p, z, F64 ? nullptr : q, n, sc, 1);
    ++res->launches;
  }
  const double bb = hsc[S_BB];
  double rel = 1.0, best = 1.0;
  int last_gain = 0;
  res->status = FE_ERR_NOT_CONVERGED;
  if (st == FE_OK && !(bb > 0.0)) {
    res->status = isfinite(bb) ? FE_OK : FE_ERR_NAN;
    rel = 0.0;
  }
  for (int it = 1; st == FE_OK && !res->handed_off && res->status == FE_ERR_NOT_CONVERGED &&
                   it <= maxit; ++it) {
    if ((st = apply(p, q)) != FE_OK) break;
    k_fcg_pq<VT><<<kRB, kT, 0, s>>>(p, q, r, mask, n, part0, part1);
    k_fcg_finish<<<1, kRB, 0, s>>>(part0, part1, sc, 1);
    k_fcg_xr<VT><<<kRB, kT, 0, s>>>(x, r, p, q, n, sc, part0, part1);
    k_fcg_finish<<<1, kRB, 0, s>>>(part0, part1, sc, 2);
    res->launches += 5;
    take_snap(it);
    if ((st = precond()) != FE_OK) break;
    k_fcg_zq<VT><<<kRB, kT, 0, s>>>(z, q, r, n, part0, part1);
    k_fcg_finish<<<1, kRB, 0, s>>>(part0, part1, sc, 3);
    res->launches += 2;
    if ((st = read_sc()) != FE_OK) break;
    res->iters = it;
    rel = sqrt(hsc[S_RR] / bb);
    if (!isfinite(rel) || !isfinite(hsc[S_PQ])) {
      res->status = FE_ERR_NAN;
      break;
    }
    if (!(hsc[S_PQ] > 0.0)) {
      res->status = FE_ERR_BREAKDOWN;
      break;
    }
    if (rel <= rtol) {
      res->status = FE_OK;
      break;
    }
    if (rel < 0.99 * best) {
      best = rel;
      last_gain = it;
    } else if (rel < best) {
      best = rel;
    }
    bool restart = false;
    if (learned && (!(hsc[S_ZR] > 0.0) || it - last_gain >= kStall || rel > 1e4 * best)) {
      learned = false;  // fall back to Jacobi from the current iterate
      restart = true;
      ++res->restarts;
      last_gain = it;
      if (res->stop_at_fallback) {
        res->handed_off = true;
        break;
      }
      if ((st = precond()) != FE_OK) break;
    }
    k_fcg_p<VT><<<kRB, kT, 0, s>>>(p, z, F64 ? nullptr : q, n, sc, restart ? 1 : 0);
    ++res->launches;
  }
  res->rel = rel;
  if constexpr (F64) {
    if (st == FE_OK) {  // true residual with the FP64 operator (FP64 data and arithmetic)
      if ((st = true_apply(x, q)) == FE_OK) {
        k_fcg_resid<<<kRB, kT, 0, s>>>(b, q, mask, n, part0, part1);
        k_fcg_finish<<<1, kRB, 0, s>>>(part0, part1, sc, 4);
        res->launches += 3;
        if ((st = read_sc()) == FE_OK)
          res->true_rel = hsc[S_BB] > 0.0 ? sqrt(hsc[S_TRUE] / hsc[S_BB]) : 0.0;
      }
    }
  }
  if (!work) cudaFree(vec);
  if (!red_in) cudaFree(red);
  return st;
}

// FCG on a single-order handle: its operator (the handle's variant; FP32 data on float vectors),
// lpc's preconditioner or Jacobi (lpc == nullptr), the FP64 operator for the true residual.
template <class VT>
int fcg_run(fe_pa* pa, int op, fe_lpc* lpc, const VT* dinv, const VT* b, VT* x, double rtol,
            int maxit, Snapshots* snap, cudaStream_t s, FcgResult* res, VT* work = nullptr,
            double* red_in = nullptr) {
  constexpr bool F64 = std::is_same<VT, double>::value;
  const fe_mesh* m = pa->mesh;
  std::function<int(const VT*, VT*)> apply = [&](const VT* in, VT* out) -> int {
    if constexpr (F64)
      return apply_dispatch(pa, op, pa->variant, in, out, s);
    else
      return apply_f32_vectors(pa, op, in, out, s, nullptr, nullptr);  // out zeroed by k_fcg_p
  };
  std::function<int(const VT*, VT*)> prec;
  if (lpc) {
    prec = [&](const VT* r, VT* z) -> int {
      if constexpr (F64)
        return fe::lpc_apply(lpc, r, z, s);
      else
        return lpc_apply32(lpc, r, z, s);
    };
  }
  std::function<int(const double*, double*)> true_apply = [&](const double* in, double* out) {
    return apply_dispatch(pa, op, FE_VARIANT_F64, in, out, s);
  };
  return fcg_core<VT>(m->ndofs, m->d_mask, m->d_map, apply, prec, true_apply, dinv, b, x, rtol,
                      maxit, snap, s, res, work, red_in);
}

// r = (1-m)(b - q) into rout; partials ||r||^2 and ||(1-m) b||^2 (the outer residual of fe_fcg_ir)
__global__ void __launch_bounds__(kT) k_ir_resid(const double* __restrict__ b,
                                                 const double* __restrict__ q,
                                                 const uint8_t* __restrict__ mask,
                                                 double* __restrict__ rout, int64_t n,
                                                 double* part0, double* part1) {
  double a = 0.0, c = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const bool bnd = mask[i] != 0;
    const double bi = bnd ? 0.0 : b[i];
    const double ri = bnd ? 0.0 : bi - q[i];
    rout[i] = ri;
    a = fma(ri, ri, a);
    c = fma(bi, bi, c);
  }
  block_partial2(a, c, part0, part1);
}

__global__ void k_add_f64(double* __restrict__ x, const double* __restrict__ d, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] += d[i];
}

// b = a * 2^shift rounded to float (the power-of-two scale is exact in FP64)
__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n,
                         int shift) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = __double2float_rn(ldexp(a[i], shift));
}

// x += d * 2^shift (exact widening and scaling by integer manipulation)
__global__ void k_add_f32(double* __restrict__ x, const float* __restrict__ d, int64_t n,
                          int shift) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] += fe::f64_from_f32_scaled(d[i], shift);
}

// Training data (first call of fe_lpc_train): probing, Cholesky, residual snapshots, samples.
// With xd/td given, also returns device FP64 copies of the pairs ([nsamp][din], caller frees)
// and the sampled elements (row r belongs to elems[r / reps]).
int make_samples(fe_lpc* L, int reps, cudaStream_t s, double** xd = nullptr,
                 double** td = nullptr, std::vector<int32_t>* elems = nullptr) {
  fe_mesh* m = const_cast<fe_mesh*>(L->pa->mesh);
  const int din = L->din;
  // Interior elements in 27 classes by (ex, ey, ez) mod 3: elements of one class are three apart,
  // so their blocks share no dof and no element and one class is probed with D^3 applies.
  // Classes are taken in turn until the block storage bound is reached.
  const int64_t cap = kProbeDoubles / ((int64_t)din * din);
  std::vector<int32_t> el;
  std::vector<int> cls_start{0};
  for (int oz = 1; oz <= 3; ++oz)
    for (int oy = 1; oy <= 3; ++oy)
      for (int ox = 1; ox <= 3; ++ox) {
        std::vector<int32_t> c;
        for (int ez = oz; ez + 1 < m->nz; ez += 3)
          for (int ey = oy; ey + 1 < m->ny; ey += 3)
            for (int ex = ox; ex + 1 < m->nx; ex += 3)
              c.push_back((int32_t)(ex + (int64_t)m->nx * (ey + (int64_t)m->ny * ez)));
        if (c.empty()) continue;
        const int64_t room = cap - (int64_t)el.size();
        if (room <= 0) break;
        if ((int64_t)c.size() > room) {  // an evenly strided subset of the class
          std::vector<int32_t> sub;
          for (int64_t i = 0; i < room; ++i) sub.push_back(c[(size_t)(i * (int64_t)c.size() / room)]);
          c.swap(sub);
        }
        el.insert(el.end(), c.begin(), c.end());
        cls_start.push_back((int)el.size());
      }
  if (el.empty())
    return set_error(FE_ERR_ARG, "fe_lpc_train: mesh too small (needs >= 3 elements per axis)");
  const int ns = (int)el.size();
  // probe applies with an FP64-accurate operator: the handle's float-float one when selected
  const int hi = (L->pa->variant == FE_VARIANT_F32X2) ? FE_VARIANT_F32X2 : FE_VARIANT_F64;
  int32_t* d_el = nullptr;
  double *v = nullptr, *w = nullptr, *Aee = nullptr, *snapbuf = nullptr;
  int* d_fail = nullptr;
  Snapshots snap;
  snap.at = {0, 1, 2, 4, 8, 16, 32, 64};
  const int nsnap = 2 * (int)snap.at.size();  // two right-hand sides
  cudaError_t err;
  const size_t mat = (size_t)ns * din * din;
  if ((err = cudaMalloc(&d_el, sizeof(int32_t) * ns)) != cudaSuccess ||
      (err = cudaMalloc(&v, sizeof(double) * m->ndofs)) != cudaSuccess ||
      (err = cudaMalloc(&w, sizeof(double) * m->ndofs)) != cudaSuccess ||
      (err = cudaMalloc(&Aee, sizeof(double) * mat)) != cudaSuccess ||
      (err = cudaMalloc(&snapbuf, sizeof(double) * nsnap * ns * din)) != cudaSuccess ||
      (err = cudaMalloc(&d_fail, sizeof(int))) != cudaSuccess) {
    cudaFree(d_el); cudaFree(v); cudaFree(w); cudaFree(Aee); cudaFree(snapbuf); cudaFree(d_fail);
    return cuda_error(err, "fe_lpc_train: sample cudaMalloc");
  }
  int st = FE_OK;
  cudaMemcpyAsync(d_el, el.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, s);
  // snapshots a short run never reaches stay zero (zero rows add nothing to loss or gradient)
  cudaMemsetAsync(snapbuf, 0, sizeof(double) * nsnap * ns * din, s);
  cudaMemsetAsync(d_fail, 0, sizeof(int), s);
  for (size_t c = 0; c + 1 < cls_start.size() && st == FE_OK; ++c) {
    const int c0 = cls_start[c], nc = cls_start[c + 1] - cls_start[c];
    for (int a = 0; a < din && st == FE_OK; ++a) {
      cudaMemsetAsync(v, 0, sizeof(double) * m->ndofs, s);
      k_probe_set<<<(nc + kT - 1) / kT, kT, 0, s>>>(v, m->d_map, d_el + c0, nc, din, a);
      st = apply_dispatch(L->pa, L->op, hi, v, w, s);
      if (st != FE_OK) break;
      k_probe_get<<<(unsigned int)(((int64_t)nc * din + kT - 1) / kT), kT, 0, s>>>(
          w, m->d_map, d_el + c0, nc, din, a, Aee + (int64_t)c0 * din * din);
    }
  }
  // residual snapshots of Jacobi-FCG on the sine load and on a random right-hand side
  snap.elems = d_el;
  snap.ns = ns;
  snap.din = din;
  for (int rhs = 0; rhs < 2 && st == FE_OK; ++rhs) {
    if (rhs == 0)
      st = fe_load_vector_sine(L->pa, v, s);
    else
      k_normal_vec<<<grid1(m->ndofs), kT, 0, s>>>(v, m->ndofs, L->seed ^ 0x5DEECE66Dull);
    if (st != FE_OK) break;
    snap.out = snapbuf + (int64_t)rhs * snap.at.size() * ns * din;
    FcgResult fr;
    st = fcg_run(L->pa, L->op, nullptr, L->dinv, v, w, 0.0, snap.at.back(), &snap, s, &fr);
  }
  if (st == FE_OK) {
    const size_t shm = sizeof(double) * din * din;
    if (shm <= 200 * 1024) {  // the whole block in shared memory (orders 1..4)
      cudaFuncSetAttribute(k_cholesky, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
      k_cholesky<<<ns, 128, shm, s>>>(Aee, din, d_fail);
    } else {                  // panels in shared memory (orders 5..8)
      const size_t pshm = sizeof(double) * din * kPanel;
      cudaFuncSetAttribute(k_cholesky_blocked, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)pshm);
      k_cholesky_blocked<<<ns, 256, pshm, s>>>(Aee, din, d_fail);
    }
    L->nsamp = (int64_t)ns * reps;
    if ((err = cudaMalloc(&L->Xs, sizeof(__nv_bfloat16) * L->nsamp * din)) != cudaSuccess ||
        (err = cudaMalloc(&L->Ts, sizeof(float) * L->nsamp * din)) != cudaSuccess)
      st = cuda_error(err, "fe_lpc_train: sample cudaMalloc");
  }
  double *Xd = nullptr, *Td = nullptr;
  if (st == FE_OK && xd) {
    if ((err = cudaMalloc(&Xd, sizeof(double) * L->nsamp * din)) != cudaSuccess ||
        (err = cudaMalloc(&Td, sizeof(double) * L->nsamp * din)) != cudaSuccess)
      st = cuda_error(err, "fe_lpc_sample_pairs: cudaMalloc");
  }
  if (st == FE_OK) {
    k_samples<<<ns, 64, sizeof(double) * 3 * din, s>>>(Aee, snapbuf, nsnap, m->d_map, d_el,
                                                       L->dis, L->wsq, ns, din, reps, L->seed,
                                                       L->Xs, L->Ts, Xd, Td);
    int fail = 0;
    if ((err = cudaGetLastError()) != cudaSuccess ||
        (err = cudaMemcpyAsync(&fail, d_fail, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (err = cudaStreamSynchronize(s)) != cudaSuccess)
      st = cuda_error(err, "fe_lpc_train: samples");
    else if (fail)
      st = set_error(FE_ERR_BREAKDOWN, "fe_lpc_train: an element block is not positive definite");
  }
  if (st != FE_OK) L->nsamp = 0;
  if (st == FE_OK && xd) {
    *xd = Xd;
    *td = Td;
    if (elems) *elems = el;
  } else {
    cudaFree(Xd);
    cudaFree(Td);
  }
  cudaFree(d_el); cudaFree(v); cudaFree(w); cudaFree(Aee); cudaFree(snapbuf); cudaFree(d_fail);
  return st;
}

}  // namespace

namespace {

constexpr size_t kMaxSmem = 232448;  // 227 KB per block (opt-in)

template <int DP, int W, class VT>
cudaError_t fused_launch(const fe_lpc* L, const VT* r, VT* z, int grid, cudaStream_t s) {
  if constexpr (mlp::FusedLayout<DP, W>::SMEM <= kMaxSmem) {
    const fe_mesh* m = L->pa->mesh;
    mlp::k_lpc_fused<DP, W, VT><<<grid, 256, mlp::FusedLayout<DP, W>::SMEM, s>>>(
        reinterpret_cast<const uint4*>(L->wimg), r, m->d_map, L->fsc32, m->ne, L->din, z);
    return cudaGetLastError();
  }
  return cudaErrorInvalidConfiguration;
}

// Blocks per SM of the fused kernel for (DP, W), 0 if it is not built or does not fit.
template <int DP, int W, class VT = double>
int fused_occupancy() {
  if constexpr (mlp::FusedLayout<DP, W>::SMEM <= kMaxSmem) {
    const int smem = (int)mlp::FusedLayout<DP, W>::SMEM;
    if (cudaFuncSetAttribute(mlp::k_lpc_fused<DP, W, VT>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
      return 0;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, mlp::k_lpc_fused<DP, W, VT>, 256,
                                                      smem) != cudaSuccess)
      return 0;
    return occ;
  }
  return 0;
}

// The built (DP, W) pairs of the fused kernel.
#define FE_FUSED_CASES(X) \
  X(16, 0) X(16, 64) X(16, 128) X(16, 256) X(32, 0) X(32, 64) X(32, 128) X(32, 256) X(64, 0) \
  X(64, 64) X(64, 128) X(64, 256) X(128, 0) X(128, 64) X(128, 128)

int fused_occ(int DP, int W) {
#define FE_OCC_CASE(dp, w) \
  if (DP == dp && W == w) return fused_occupancy<dp, w>();
  FE_FUSED_CASES(FE_OCC_CASE)
#undef FE_OCC_CASE
  return 0;
}

cudaError_t fused_run(const fe_lpc* L, const double* r, double* z, cudaStream_t s) {
  const int DP = mlp::fused_dp(L->din), W = L->width;
#define FE_RUN_CASE(dp, w) \
  if (DP == dp && W == w) return fused_launch<dp, w, double>(L, r, z, L->fused_grid, s);
  FE_FUSED_CASES(FE_RUN_CASE)
#undef FE_RUN_CASE
  return cudaErrorInvalidConfiguration;
}

// FP32 vectors (the mixed-precision inner solve): the linear map and widths 64, 128.
#define FE_FUSED_CASES_F32(X) \
  X(16, 0) X(32, 0) X(64, 0) X(128, 0) X(16, 64) X(32, 64) X(64, 64) X(128, 64) X(16, 128) \
  X(32, 128) X(64, 128) X(128, 128)

bool fused_f32_built(const fe_lpc* L) {
  const int DP = mlp::fused_dp(L->din), W = L->width;
#define FE_HAS_CASE(dp, w) \
  if (DP == dp && W == w) return true;
  FE_FUSED_CASES_F32(FE_HAS_CASE)
#undef FE_HAS_CASE
  return false;
}

cudaError_t fused_run_f32(const fe_lpc* L, const float* r, float* z, cudaStream_t s) {
  const int DP = mlp::fused_dp(L->din), W = L->width;
#define FE_RUN_CASE32(dp, w)                                                               \
  if (DP == dp && W == w) {                                                               \
    static bool attr = fused_occupancy<dp, w, float>() > 0;                               \
    return attr ? fused_launch<dp, w, float>(L, r, z, L->fused_grid, s)                   \
                : cudaErrorInvalidConfiguration;                                          \
  }
  FE_FUSED_CASES_F32(FE_RUN_CASE32)
#undef FE_RUN_CASE32
  return cudaErrorInvalidConfiguration;
}

// Chooses the fused kernel when one is built for (D^3, width) and fits in shared memory.
void fused_setup(fe_lpc* L) {
  L->fused_grid = 0;
  const int DP = mlp::fused_dp(L->din);
  const int occ = fused_occ(DP, L->width);
  if (occ <= 0) return;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return;
  int64_t off[5];
  mlp::fused_offsets(DP, L->width, off);
  if (cudaMalloc(&L->wimg, sizeof(__nv_bfloat16) * off[4]) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  const int64_t tiles = (L->pa->mesh->ne + 15) / 16;
  const int64_t want = (tiles + 7) / 8;
  const int64_t cap = (int64_t)sms * occ;
  L->fused_grid = (int)(want < cap ? (want < 1 ? 1 : want) : cap);
}

// ---- the tcgen05 fused apply (fe_mlp_tc.cuh)
constexpr int kSmemPerSm = 233472;  // 228 KB of shared memory per SM

// Dynamic shared memory per CTA: the layout's, raised where needed so that no more CTAs fit on
// one SM than its 512 TMEM columns serve (a CTA whose allocation cannot be met would otherwise
// wait inside tcgen05.alloc for another CTA to finish).
template <int DP, int W>
constexpr int tc_smem() {
  using Lay = typename mlptc::TcConfig<DP, W>::Lay;
  constexpr int cap = 512 / Lay::NCOLS;
  constexpr int floor_ = kSmemPerSm / (cap + 1) + 1;
  return Lay::SMEM > floor_ ? Lay::SMEM : floor_;
}

template <int DP, int W, class VT>
constexpr auto tc_kernel() {
  using C = mlptc::TcConfig<DP, W>;
  return mlptc::k_lpc_tc<DP, W, VT, C::G, C::AT, C::WPG>;
}

// Resident CTAs per SM of the tcgen05 apply for (DP, W), 0 if it does not fit.
template <int DP, int W, class VT>
int tc_occupancy() {
  using C = mlptc::TcConfig<DP, W>;
  constexpr int smem = tc_smem<DP, W>();
  if constexpr (C::FITS && smem <= (int)kMaxSmem) {
    auto kern = tc_kernel<DP, W, VT>();
    int occ = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, C::THREADS, smem) !=
            cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    const int cap = 512 / C::Lay::NCOLS;
    return occ < cap ? occ : cap;
  }
  return 0;
}

template <int DP, int W, class VT>
cudaError_t tc_launch(const fe_lpc* L, const VT* r, VT* z, int grid, cudaStream_t s) {
  using C = mlptc::TcConfig<DP, W>;
  constexpr int smem = tc_smem<DP, W>();
  if constexpr (C::FITS && smem <= (int)kMaxSmem) {
    const fe_mesh* m = L->pa->mesh;
    tc_kernel<DP, W, VT>()<<<grid, C::THREADS, smem, s>>>(L->tcimg, r, m->d_map, L->fsc32, m->ne,
                                                         L->din, z, L->d_tcfail);
    return cudaGetLastError();
  }
  return cudaErrorInvalidConfiguration;
}

// Tile pipelines per CTA of the built (DP, W) (the grid counts pairs of tiles where it is 2).
int tc_groups_of(int DP, int W);

// The built (DP, W) pairs of the tcgen05 apply.
#define FE_TC_CASES(X) \
  X(16, 0) X(16, 64) X(16, 128) X(16, 256) X(32, 0) X(32, 64) X(32, 128) X(32, 256) X(64, 0) \
  X(64, 64) X(64, 128) X(64, 256) X(128, 0) X(128, 64) X(128, 128)

int tc_groups_of(int DP, int W) {
#define FE_TC_G(dp, w) \
  if (DP == dp && W == w) return mlptc::TcConfig<dp, w>::G;
  FE_TC_CASES(FE_TC_G)
#undef FE_TC_G
  return 1;
}

template <class VT>
int tc_occ(int DP, int W) {
#define FE_TC_OCC(dp, w) \
  if (DP == dp && W == w) return tc_occupancy<dp, w, VT>();
  FE_TC_CASES(FE_TC_OCC)
#undef FE_TC_OCC
  return 0;
}

template <class VT>
cudaError_t tc_run(const fe_lpc* L, const VT* r, VT* z, int grid, cudaStream_t s) {
  const int DP = mlp::fused_dp(L->din), W = L->width;
#define FE_TC_RUN(dp, w) \
  if (DP == dp && W == w) return tc_launch<dp, w, VT>(L, r, z, grid, s);
  FE_TC_CASES(FE_TC_RUN)
#undef FE_TC_RUN
  return cudaErrorInvalidConfiguration;
}

// Persistent grids of the tcgen05 apply for FP64 and FP32 vectors (0 where it is not built or
// the device has no tcgen05), its weight images and its fault flag.
void tc_setup(fe_lpc* L) {
  L->tc_grid = L->tc_grid32 = 0;
  int dev = 0, sms = 0, major = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  if (major != 10) return;  // tcgen05: the sm_100 family
  const int DP = mlp::fused_dp(L->din);
  const int occ = tc_occ<double>(DP, L->width), occ32 = tc_occ<float>(DP, L->width);
  if (occ <= 0 && occ32 <= 0) return;
  int64_t off[5];
  mlptc::tc_offsets(DP, L->width, off);
  if (cudaMalloc(&L->tcimg, sizeof(__nv_bfloat16) * off[4]) != cudaSuccess ||
      cudaMalloc(&L->d_tcfail, sizeof(int)) != cudaSuccess ||
      cudaMemset(L->d_tcfail, 0, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(L->tcimg);
    cudaFree(L->d_tcfail);
    L->tcimg = nullptr;
    L->d_tcfail = nullptr;
    return;
  }
  // one CTA runs G pipelines on interleaved 128-element tiles
  const int64_t tiles = (L->pa->mesh->ne + mlptc::kRows - 1) / mlptc::kRows;
  const int G = tc_groups_of(DP, L->width);
  const int64_t units = (tiles + G - 1) / G;
  auto grid = [&](int o) -> int {
    if (o <= 0) return 0;
    const int64_t cap = (int64_t)sms * o;
    return (int)(units < cap ? (units < 1 ? 1 : units) : cap);
  };
  L->tc_grid = grid(occ);
  L->tc_grid32 = grid(occ32);
}

// The inference kernel a call uses (AUTO resolved); fp32: the FP32-vector solves, which have
// no unfused path.  AUTO takes the measured-fastest built kernel: tcgen05 at width 256, where
// the layers are dense enough for the tensor cores to matter; below that the mma.sync fused
// kernel (its independent 16-element warps hide the dof-map gather's latency as well as the
// tcgen05 tile pipelines do at width 128, and better for the linear map); else whichever fused
// kernel is built; else the GEMMs.
int lpc_kernel(const fe_lpc* L, bool fp32) {
  if (L->kernel != FE_LPC_KERNEL_AUTO) return L->kernel;
  const bool tc = (fp32 ? L->tc_grid32 : L->tc_grid) > 0;
  const bool ms = L->fused_grid > 0 && (!fp32 || fused_f32_built(L));
  if (tc && (L->width >= 256 || !ms)) return FE_LPC_KERNEL_TCGEN05;
  if (ms) return FE_LPC_KERNEL_MMA_SYNC;
  return FE_LPC_KERNEL_GEMM;
}

// The tcgen05 weight images, packed on first use after every weight update.
void tc_pack(fe_lpc* L, cudaStream_t s) {
  if (L->tcimg_ok) return;
  int64_t off[5];
  const int DP = mlp::fused_dp(L->din);
  mlptc::tc_offsets(DP, L->width, off);
  mlptc::k_pack_tc<<<grid1(off[4]), kT, 0, s>>>(L->w32, L->din, L->width, DP, L->tcimg);
  L->tcimg_ok = true;
}

// 1 if a tcgen05 launch has given up a wait (synchronous read of the device flag).
int tc_faulted(const fe_lpc* L) {
  if (!L || !L->d_tcfail) return 0;
  int f = 0;
  if (cudaMemcpy(&f, L->d_tcfail, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
  return f;
}

}  // namespace

namespace {
// z = M(r) on FP32 vectors with the fused kernel (z overwritten).
int lpc_apply32(fe_lpc* L, const float* r, float* z, cudaStream_t s) {
  cudaError_t err;
  if ((err = cudaMemsetAsync(z, 0, sizeof(float) * L->pa->mesh->ndofs, s)) != cudaSuccess)
    return cuda_error(err, "fe_fcg_ir: zero z");
  if (lpc_kernel(L, true) == FE_LPC_KERNEL_TCGEN05) {
    tc_pack(L, s);
    return cuda_error(tc_run<float>(L, r, z, L->tc_grid32, s), "fe_fcg_ir: tcgen05 launch");
  }
  if (!L->wimg_ok) {
    int64_t off[5];
    const int DP = mlp::fused_dp(L->din);
    mlp::fused_offsets(DP, L->width, off);
    mlp::k_pack_wimg<<<grid1(off[4]), kT, 0, s>>>(L->w32, L->din, L->width, DP, L->wimg);
    L->wimg_ok = true;
  }
  return cuda_error(fused_run_f32(L, r, z, s), "fe_fcg_ir: fused launch");
}
}  // namespace

namespace fe {
// z = M(r): the learned additive patch preconditioner (z overwritten, or z += M(r) when
// accumulating).
int lpc_apply(fe_lpc* L, const double* r, double* z, cudaStream_t s, bool accumulate) {
  const fe_mesh* m = L->pa->mesh;
  const int din = L->din;
  const int kernel = lpc_kernel(L, false);
  if (kernel == FE_LPC_KERNEL_TCGEN05) {
    cudaError_t err;
    if (!accumulate && (err = cudaMemsetAsync(z, 0, sizeof(double) * m->ndofs, s)) != cudaSuccess)
      return cuda_error(err, "fe_lpc_apply: zero z");
    tc_pack(L, s);
    return cuda_error(tc_run<double>(L, r, z, L->tc_grid, s), "fe_lpc_apply: tcgen05 launch");
  }
  if (kernel == FE_LPC_KERNEL_MMA_SYNC) {
    cudaError_t err;
    if (!accumulate && (err = cudaMemsetAsync(z, 0, sizeof(double) * m->ndofs, s)) != cudaSuccess)
      return cuda_error(err, "fe_lpc_apply: zero z");
    const int DP = mlp::fused_dp(din);
    if (!L->wimg_ok) {
      int64_t off[5];
      mlp::fused_offsets(DP, L->width, off);
      mlp::k_pack_wimg<<<grid1(off[4]), kT, 0, s>>>(L->w32, din, L->width, DP, L->wimg);
      L->wimg_ok = true;
    }
    return cuda_error(fused_run(L, r, z, s), "fe_lpc_apply: fused launch");
  }
  const int64_t chunk = m->ne < (1 << 18) ? m->ne : (1 << 18);  // rows per pass
  int st = ensure_workspace(L, chunk);
  if (st != FE_OK) return st;
  cudaError_t err;
  if (!accumulate && (err = cudaMemsetAsync(z, 0, sizeof(double) * m->ndofs, s)) != cudaSuccess)
    return cuda_error(err, "fe_lpc_apply: zero z");
  for (int64_t e0 = 0; e0 < m->ne; e0 += chunk) {
    const int64_t rows = (m->ne - e0) < chunk ? (m->ne - e0) : chunk;
    k_lpc_gather<<<(unsigned int)((rows + 7) / 8), 256, 0, s>>>(r, m->d_map, L->fsc, e0, rows, din,
                                                               L->Xb, L->scale);
    if ((st = mlp_forward(L, rows, s, false)) != FE_OK) return st;
    k_lpc_scatter<<<(unsigned int)((rows * din + kT - 1) / kT), kT, 0, s>>>(L->Y, L->scale, m->d_map,
                                                                           L->fsc, e0, rows, din, z);
  }
  return cuda_error(cudaGetLastError(), "fe_lpc_apply launch");
}

int fcg_solve(const FcgOperator& op, const double* dinv, const double* b, double* x, double rtol,
              int maxit, cudaStream_t s, fe_pcg_stats* stats, const char* who) {
  const auto t0 = std::chrono::steady_clock::now();
  FcgResult res;
  const int st = fcg_core<double>(op.n, op.mask, nullptr, op.apply, op.prec, op.true_apply, dinv,
                                  b, x, rtol, maxit, nullptr, s, &res);
  if (st != FE_OK) return st;
  if (stats) {
    stats->iters = res.iters;
    stats->rel_resid = res.rel;
    stats->true_rel_resid = res.true_rel;
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    stats->launches = res.launches;
    stats->outer_iters = 1 + res.restarts;
  }
  switch (res.status) {
    case FE_OK:
      return FE_OK;
    case FE_ERR_BREAKDOWN:
      return set_error(FE_ERR_BREAKDOWN, std::string(who) + ": p.Ap <= 0");
    case FE_ERR_NAN:
      return set_error(FE_ERR_NAN, std::string(who) + ": NaN or Inf in the iteration");
    default:
      return set_error(FE_ERR_NOT_CONVERGED, std::string(who) + ": maxit reached before rtol");
  }
}

// Order, patch size D^3 and width of a handle.
void lpc_shape(const fe_lpc* L, int* order, int* din, int* width) {
  if (order) *order = L->pa->p;
  if (din) *din = L->din;
  if (width) *width = L->width;
}

// dst's weights := src's (same patch size and width); the inference images are rebuilt on use.
int lpc_copy_weights(fe_lpc* dst, const fe_lpc* src, cudaStream_t s) {
  if (dst->din != src->din || dst->width != src->width)
    return set_error(FE_ERR_ARG, "learned preconditioner: patch size or width differ");
  cudaError_t err = cudaMemcpyAsync(dst->w32, src->w32, 4 * (size_t)src->nparam,
                                    cudaMemcpyDeviceToDevice, s);
  if (err != cudaSuccess) return cuda_error(err, "learned preconditioner: weight copy");
  k_to_bf16<<<grid1(dst->nparam), kT, 0, s>>>(dst->w32, dst->wb, dst->nparam);
  dst->wimg_ok = false;
  dst->tcimg_ok = false;
  return cuda_error(cudaGetLastError(), "learned preconditioner: weight copy");
}

// The input/output scaling F of the patch operator (FP64 [ndofs], 0 on masked dofs) replaced by
// a caller's (the shared scaling of a variable-order space).
int lpc_set_scaling(fe_lpc* L, const double* F, cudaStream_t s) {
  const int64_t n = L->pa->mesh->ndofs;
  cudaError_t err = cudaMemcpyAsync(L->fsc, F, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
  if (err != cudaSuccess) return cuda_error(err, "learned preconditioner: scaling");
  k_to_f32<<<grid1(n), kT, 0, s>>>(L->fsc, L->fsc32, n, 0);
  return cuda_error(cudaGetLastError(), "learned preconditioner: scaling");
}
}  // namespace fe

extern "C" {

int fe_fcg_ir(fe_pa* pa, int op, fe_lpc* lpc, const double* dev_b, double* dev_x, double rtol,
              int maxit, double inner_rtol, fe_pcg_stats* stats, void* stream) {
  clear_error();
  const auto t0 = std::chrono::steady_clock::now();
  if (stats) *stats = fe_pcg_stats{0, 0.0, 0.0, 0.0, 0, 0};
  if (!pa || !lpc || !dev_b || !dev_x) return set_error(FE_ERR_ARG, "fe_fcg_ir: null argument");
  if (op != FE_DIFFUSION && op != FE_MASS) return set_error(FE_ERR_ARG, "fe_fcg_ir: bad op");
  if (!(pa->ops & op)) return set_error(FE_ERR_ARG, "fe_fcg_ir: operator not set up");
  if (lpc->pa != pa || lpc->op != op)
    return set_error(FE_ERR_ARG, "fe_fcg_ir: preconditioner built for another operator");
  if (maxit < 1 || !(rtol >= 0.0)) return set_error(FE_ERR_ARG, "fe_fcg_ir: bad rtol or maxit");
  if (inner_rtol == 0.0) inner_rtol = 1e-2;
  if (!(inner_rtol > 0.0 && inner_rtol < 1.0))
    return set_error(FE_ERR_ARG, "fe_fcg_ir: inner_rtol must lie in (0, 1)");
  {
    const int k = lpc_kernel(lpc, true);
    const bool ok = (k == FE_LPC_KERNEL_TCGEN05 && lpc->tc_grid32 > 0) ||
                    (k == FE_LPC_KERNEL_MMA_SYNC && lpc->fused_grid > 0 && fused_f32_built(lpc));
    if (!ok)
      return set_error(FE_ERR_UNSUPPORTED,
                       "fe_fcg_ir: no FP32 fused kernel for this order, width and kernel choice");
  }
  cudaStream_t s = (cudaStream_t)stream;
  int st;
  if ((op == FE_DIFFUSION ? pa->d_qd_diff32 : pa->d_qd_mass32) == nullptr) {
    const int saved = pa->variant;
    if ((st = fe_pa_set_variant(pa, FE_VARIANT_F32, stream)) != FE_OK) return st;
    pa->variant = saved;
  }
  // The outer residual is FP64 (FP64 data and arithmetic).  The inner solves run on
  // A32 = 2^-s A (the FP32 data carry the shift s that puts them in the float range) with the
  // right-hand side r 2^-e (e the exponent of ||r||, so that it stays in the float range as the
  // refinement shrinks r); their solution d32 = A32^-1 r 2^-e gives d = 2^(e - s) d32.
  const int qs = pa->qd32_shift[op == FE_DIFFUSION ? 0 : 1];
  const fe_mesh* m = pa->mesh;
  const int64_t n = m->ndofs;
  double *dv = nullptr, *red = nullptr;
  float* fv = nullptr;
  cudaError_t err;
  if ((err = cudaMalloc(&dv, sizeof(double) * 2 * n)) != cudaSuccess ||
      (err = cudaMalloc(&red, sizeof(double) * (2 * kRB + S_N))) != cudaSuccess ||
      (err = cudaMalloc(&fv, sizeof(float) * 7 * n)) != cudaSuccess) {
    cudaFree(dv);
    cudaFree(red);
    return cuda_error(err, "fe_fcg_ir: cudaMalloc");
  }
  double *rr = dv, *q = dv + n;
  float *r32 = fv, *x32 = fv + n, *d32 = fv + 2 * n, *work32 = fv + 3 * n;
  double *part0 = red, *part1 = red + kRB, *sc = red + 2 * kRB;
  int launches = 0, outer = 0, inner_total = 0, restarts = 0;
  double rel = 1.0, rnorm = 0.0;
  auto outer_residual = [&]() -> int {  // rr = (1-m)(b - A x) with the FP64 operator
    int st2 = apply_dispatch(pa, op, FE_VARIANT_F64, dev_x, q, s);
    if (st2 != FE_OK) return st2;
    k_ir_resid<<<kRB, kT, 0, s>>>(dev_b, q, m->d_mask, rr, n, part0, part1);
    k_fcg_finish<<<1, kRB, 0, s>>>(part0, part1, sc, 4);
    launches += 3;
    double hsc[S_N];
    cudaError_t e;
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(hsc, sc, sizeof(hsc), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
      return cuda_error(e, "fe_fcg_ir: residual");
    rel = hsc[S_BB] > 0.0 ? sqrt(hsc[S_TRUE] / hsc[S_BB]) : 0.0;
    rnorm = sqrt(hsc[S_TRUE]);
    return FE_OK;
  };
  int state = FE_ERR_NOT_CONVERGED;
  st = cuda_error(cudaMemsetAsync(dev_x, 0, sizeof(double) * n, s), "fe_fcg_ir: zero x");
  if (st == FE_OK) {
    k_to_f32<<<grid1(n), kT, 0, s>>>(lpc->dinv, d32, n, qs);  // inverse diagonal of A32
    ++launches;
    st = outer_residual();
  }
  if (st == FE_OK && rel <= rtol) state = FE_OK;
  while (st == FE_OK && state == FE_ERR_NOT_CONVERGED) {
    if (!std::isfinite(rel)) {
      state = FE_ERR_NAN;
      break;
    }
    int e = 0;
    std::frexp(rnorm, &e);
    k_to_f32<<<grid1(n), kT, 0, s>>>(rr, r32, n, -e);
    ++launches;
    FcgResult in;
    st = fcg_run<float>(pa, op, lpc, d32, r32, x32, inner_rtol, maxit - inner_total, nullptr, s,
                        &in, work32, red);
    if (st != FE_OK) break;
    launches += in.launches;
    inner_total += in.iters;
    restarts += in.restarts;
    ++outer;
    if (in.status == FE_ERR_NAN || in.status == FE_ERR_BREAKDOWN) {
      state = in.status;
      break;
    }
    k_add_f32<<<grid1(n), kT, 0, s>>>(dev_x, x32, n, e - qs);
    ++launches;
    const double prev = rel;
    if ((st = outer_residual()) != FE_OK) break;
    if (rel <= rtol)
      state = FE_OK;
    else if (inner_total >= maxit || !(rel < prev))
      state = FE_ERR_NOT_CONVERGED;  // budget spent, or refinement stagnated
    if (state == FE_ERR_NOT_CONVERGED && (inner_total >= maxit || !(rel < prev))) break;
  }
  cudaFree(dv);
  cudaFree(red);
  cudaFree(fv);
  if (st != FE_OK) return st;
  if (stats) {
    stats->iters = inner_total;
    stats->rel_resid = rel;
    stats->true_rel_resid = rel;
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    stats->launches = launches;
    stats->outer_iters = outer;
  }
  if (tc_faulted(lpc))
    return set_error(FE_ERR_CUDA, "fe_fcg_ir: the tcgen05 preconditioner gave up a wait on the "
                                  "tensor core");
  switch (state) {
    case FE_OK:
      return FE_OK;
    case FE_ERR_NAN:
      return set_error(FE_ERR_NAN, "fe_fcg_ir: NaN or Inf in the iteration");
    case FE_ERR_BREAKDOWN:
      return set_error(FE_ERR_BREAKDOWN, "fe_fcg_ir: p.Ap <= 0 in the inner solve");
    default:
      return set_error(FE_ERR_NOT_CONVERGED, "fe_fcg_ir: maxit reached or refinement stagnated");
  }
}

int fe_lpc_create(fe_pa* pa, int op, int width, uint64_t seed, fe_lpc** out) {
  clear_error();
  if (!out) return set_error(FE_ERR_ARG, "fe_lpc_create: out is NULL");
  *out = nullptr;
  if (!pa) return set_error(FE_ERR_ARG, "fe_lpc_create: pa is NULL");
  if (op != FE_DIFFUSION && op != FE_MASS) return set_error(FE_ERR_ARG, "fe_lpc_create: bad op");
  if (!(pa->ops & op)) return set_error(FE_ERR_ARG, "fe_lpc_create: operator not set up");
  if ((width != 0 && width < 8) || width > 4096)
    return set_error(FE_ERR_ARG, "fe_lpc_create: width must be 0 (linear) or 8..4096");
  if (pa->p > kLpcMaxOrder)
    return set_error(FE_ERR_UNSUPPORTED, "fe_lpc_create: orders above 8 are not built");
  fe_lpc* L = new fe_lpc();
  L->pa = pa;
  L->op = op;
  L->din = pa->D * pa->D * pa->D;
  L->width = width;
  L->seed = seed;
  L->nparam = 2LL * L->din * width + (int64_t)width * width + (int64_t)L->din * L->din;
  const fe_mesh* m = pa->mesh;
  cudaStream_t s = 0;
  cudaError_t err;
  if ((err = cudaMalloc(&L->w32, 4 * L->nparam)) != cudaSuccess ||
      (err = cudaMalloc(&L->wb, 2 * L->nparam)) != cudaSuccess ||
      (err = cudaMalloc(&L->adam_m, 4 * L->nparam)) != cudaSuccess ||
      (err = cudaMalloc(&L->adam_v, 4 * L->nparam)) != cudaSuccess ||
      (err = cudaMalloc(&L->grad, 4 * L->nparam)) != cudaSuccess ||
      (err = cudaMalloc(&L->wsq, 8 * m->ndofs)) != cudaSuccess ||
      (err = cudaMalloc(&L->dinv, 8 * m->ndofs)) != cudaSuccess ||
      (err = cudaMalloc(&L->dis, 8 * m->ndofs)) != cudaSuccess ||
      (err = cudaMalloc(&L->fsc, 8 * m->ndofs)) != cudaSuccess ||
      (err = cudaMalloc(&L->fsc32, 4 * m->ndofs)) != cudaSuccess ||
      (err = cudaMalloc(&L->red, 16)) != cudaSuccess) {
    fe_lpc_destroy(L);
    return cuda_error(err, "fe_lpc_create: cudaMalloc");
  }
  cudaMemsetAsync(L->adam_m, 0, 4 * L->nparam, s);
  cudaMemsetAsync(L->adam_v, 0, 4 * L->nparam, s);
  k_init_weights<<<grid1(L->nparam), kT, 0, s>>>(L->w32, L->din, width, seed);
  k_to_bf16<<<grid1(L->nparam), kT, 0, s>>>(L->w32, L->wb, L->nparam);
  cudaMemsetAsync(L->wsq, 0, 8 * m->ndofs, s);
  k_count<<<grid1(m->ne * L->din), kT, 0, s>>>(m->d_map, m->ne * L->din, L->wsq);
  k_wsq<<<grid1(m->ndofs), kT, 0, s>>>(L->wsq, m->d_mask, m->ndofs);
  int st = fe_assemble_diagonal(pa, op, L->dinv, s);
  if (st == FE_OK) {
    k_invert_diag<<<grid1(m->ndofs), kT, 0, s>>>(L->dinv, m->d_mask, m->ndofs);
    k_sqrt_vec<<<grid1(m->ndofs), kT, 0, s>>>(L->dinv, L->dis, L->wsq, L->fsc, m->ndofs);
    k_to_f32<<<grid1(m->ndofs), kT, 0, s>>>(L->fsc, L->fsc32, m->ndofs, 0);
    err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) st = cuda_error(err, "fe_lpc_create");
  }
  if (st != FE_OK) {
    fe_lpc_destroy(L);
    return st;
  }
  fused_setup(L);
  tc_setup(L);
  *out = L;
  return FE_OK;
}

}  // extern "C"

namespace {
// One Adam step (beta 0.9 / 0.999, eps 1e-8) on the gradient in L->grad; refreshes the BF16
// copy of the weights.
int adam_update(fe_lpc* L, double lr, cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  ++L->adam_t;
  const float c1 = 1.0f - powf(b1, (float)L->adam_t), c2 = 1.0f - powf(b2, (float)L->adam_t);
  L->wimg_ok = false;
  L->tcimg_ok = false;
  k_adam<<<grid1(L->nparam), kT, 0, s>>>(L->w32, L->grad, L->adam_m, L->adam_v, L->nparam,
                                         (float)lr, b1, b2, 1e-8f, c1, c2, L->wb);
  return cuda_error(cudaGetLastError(), "fe_lpc: Adam step launch");
}
}  // namespace

extern "C" {

int fe_lpc_train(fe_lpc* L, int steps, int batch, double lr, int reps, double* final_loss,
                 void* stream) {
  clear_error();
  if (!L) return set_error(FE_ERR_ARG, "fe_lpc_train: NULL handle");
  if (steps < 0 || batch < 1 || batch > (1 << 20) || !(lr > 0.0))
    return set_error(FE_ERR_ARG, "fe_lpc_train: bad steps, batch (1..2^20) or lr");
  cudaStream_t s = (cudaStream_t)stream;
  int st;
  if (L->nsamp == 0 && (st = make_samples(L, reps > 0 ? reps : 16, s)) != FE_OK) return st;
  if ((st = ensure_workspace(L, batch)) != FE_OK) return st;
  double loss = 0.0;
  for (int it = 0; it < steps; ++it) {
    const uint64_t key = L->seed * 0x9E3779B97F4A7C15ull + (uint64_t)(L->adam_t + 1) * 0x632BE59BD9B4E019ull;
    k_batch<<<(unsigned int)(((int64_t)batch * L->din + kT - 1) / kT), kT, 0, s>>>(
        L->Xs, L->Ts, L->nsamp, L->din, batch, key, L->Xb, L->Tb);
    if ((st = mlp_loss_grad(L, batch, s, (it + 1 == steps) ? &loss : nullptr)) != FE_OK) return st;
    if ((st = adam_update(L, lr, s)) != FE_OK) return st;
  }
  if (final_loss) *final_loss = loss;
  return cuda_error(cudaStreamSynchronize(s), "fe_lpc_train");
}

int fe_lpc_fit_linear(fe_lpc* L, double ridge, int reps, double* fit_loss, void* stream) {
  clear_error();
  if (!L) return set_error(FE_ERR_ARG, "fe_lpc_fit_linear: NULL handle");
  if (!(ridge >= 0.0)) return set_error(FE_ERR_ARG, "fe_lpc_fit_linear: ridge must be >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  int st;
  if (L->nsamp == 0 && (st = make_samples(L, reps > 0 ? reps : 16, s)) != FE_OK) return st;
  const int d = L->din;
  const int64_t N = L->nsamp;
  // G = X^T X, H = X^T T over all pairs (BF16 operands, FP32 accumulation), ||T||^2
  __nv_bfloat16* tb = nullptr;
  float* gh = nullptr;
  cudaError_t err;
  if ((err = cudaMalloc(&tb, sizeof(__nv_bfloat16) * N * d)) != cudaSuccess ||
      (err = cudaMalloc(&gh, sizeof(float) * 2 * d * d)) != cudaSuccess) {
    cudaFree(tb);
    return cuda_error(err, "fe_lpc_fit_linear: cudaMalloc");
  }
  k_to_bf16<<<grid1(N * d), kT, 0, s>>>(L->Ts, tb, N * d);
  cudaMemsetAsync(L->red, 0, 2 * sizeof(double), s);
  k_loss_terms<<<grid1(N * d), kT, 0, s>>>(L->Ts, L->Ts, N * d, L->red);  // red[1] = ||T||^2
  if ((err = mlp::gemm<true, false, mlp::EPI_STORE>(d, d, (int)N, L->Xs, d, L->Xs, d, gh, d,
                                                    nullptr, 0, s)) != cudaSuccess ||
      (err = mlp::gemm<true, false, mlp::EPI_STORE>(d, d, (int)N, L->Xs, d, tb, d, gh + d * d, d,
                                                    nullptr, 0, s)) != cudaSuccess) {
    cudaFree(tb);
    cudaFree(gh);
    return cuda_error(err, "fe_lpc_fit_linear: GEMM launch");
  }
  std::vector<float> hgh(2 * d * d);
  double red[2];
  err = cudaMemcpyAsync(hgh.data(), gh, sizeof(float) * 2 * d * d, cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess) err = cudaMemcpyAsync(red, L->red, sizeof(red), cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  cudaFree(tb);
  cudaFree(gh);
  if (err != cudaSuccess) return cuda_error(err, "fe_lpc_fit_linear: copy");
  // (G + ridge mean(diag G) I) W0 = H by FP64 Cholesky on the host
  std::vector<double> G(d * d), W(d * d);
  double tr = 0.0;
  for (int i = 0; i < d; ++i) tr += hgh[i * d + i];
  const double lam = ridge * tr / d;
  for (int i = 0; i < d * d; ++i) G[i] = hgh[i];
  for (int i = 0; i < d; ++i) G[i * d + i] += lam;
  for (int k = 0; k < d; ++k) {
    double dk = G[k * d + k];
    for (int j = 0; j < k; ++j) dk -= G[k * d + j] * G[k * d + j];
    if (!(dk > 0.0)) return set_error(FE_ERR_BREAKDOWN, "fe_lpc_fit_linear: singular normal equations");
    G[k * d + k] = sqrt(dk);
    for (int i = k + 1; i < d; ++i) {
      double v = G[i * d + k];
      for (int j = 0; j < k; ++j) v -= G[i * d + j] * G[k * d + j];
      G[i * d + k] = v / G[k * d + k];
    }
  }
  for (int c = 0; c < d; ++c) {  // column c of W0 from column c of H
    std::vector<double> y(d);
    for (int i = 0; i < d; ++i) {
      double v = hgh[d * d + i * d + c];
      for (int j = 0; j < i; ++j) v -= G[i * d + j] * y[j];
      y[i] = v / G[i * d + i];
    }
    for (int i = d - 1; i >= 0; --i) {
      double v = y[i];
      for (int j = i + 1; j < d; ++j) v -= G[j * d + i] * W[j * d + c];
      W[i * d + c] = v / G[i * d + i];
    }
  }
  // the map kept is the symmetric part of the fit: the local inverse it approximates is
  // symmetric, and an antisymmetric remainder (sampling noise, a few per cent) makes flexible CG
  // with one stored direction stall and fall back at high coefficient contrast
  for (int i = 0; i < d; ++i)
    for (int c = i + 1; c < d; ++c) {
      const double v = 0.5 * (W[i * d + c] + W[c * d + i]);
      W[i * d + c] = v;
      W[c * d + i] = v;
    }
  // loss = (||T||^2 - 2 tr(W^T H) + tr(W^T G W)) / ||T||^2 with the unregularised G
  double cross = 0.0, quad = 0.0;
  for (int i = 0; i < d; ++i)
    for (int c = 0; c < d; ++c) {
      cross += W[i * d + c] * hgh[d * d + i * d + c];
      double gw = 0.0;
      for (int j = 0; j < d; ++j) gw += (double)hgh[i * d + j] * W[j * d + c];
      quad += W[i * d + c] * gw;
    }
  if (fit_loss) *fit_loss = red[1] > 0.0 ? (red[1] - 2.0 * cross + quad) / red[1] : 0.0;
  // W0 is the last d x d block of the packed weights
  std::vector<float> w0(d * d);
  for (int i = 0; i < d * d; ++i) w0[i] = (float)W[i];
  const int64_t off = L->nparam - (int64_t)d * d;
  if ((err = cudaMemcpyAsync(L->w32 + off, w0.data(), sizeof(float) * d * d,
                             cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return cuda_error(err, "fe_lpc_fit_linear: weights");
  k_to_bf16<<<grid1(L->nparam), kT, 0, s>>>(L->w32, L->wb, L->nparam);
  L->wimg_ok = false;
  L->tcimg_ok = false;
  return cuda_error(cudaStreamSynchronize(s), "fe_lpc_fit_linear");
}

int fe_lpc_weights(fe_lpc* L, float* host_w, int set) {
  clear_error();
  if (!L || !host_w) return set_error(FE_ERR_ARG, "fe_lpc_weights: null argument");
  cudaError_t err;
  if (set) {
    if ((err = cudaMemcpy(L->w32, host_w, 4 * L->nparam, cudaMemcpyHostToDevice)) != cudaSuccess)
      return cuda_error(err, "fe_lpc_weights");
    k_to_bf16<<<grid1(L->nparam), kT>>>(L->w32, L->wb, L->nparam);
    L->wimg_ok = false;
    L->tcimg_ok = false;
    return cuda_error(cudaDeviceSynchronize(), "fe_lpc_weights");
  }
  return cuda_error(cudaMemcpy(host_w, L->w32, 4 * L->nparam, cudaMemcpyDeviceToHost),
                    "fe_lpc_weights");
}

int fe_lpc_loss_grad(fe_lpc* L, int batch, const float* host_x, const float* host_t,
                     float* host_y, float* host_grad, double* loss) {
  clear_error();
  if (!L || !host_x || !host_t || batch < 1 || batch > (1 << 20))
    return set_error(FE_ERR_ARG, "fe_lpc_loss_grad: bad arguments");
  int st = ensure_workspace(L, batch);
  if (st != FE_OK) return st;
  const int64_t n = (int64_t)batch * L->din;
  std::vector<__nv_bfloat16> xb(n);
  for (int64_t i = 0; i < n; ++i) xb[i] = __float2bfloat16(host_x[i]);
  cudaError_t err;
  if ((err = cudaMemcpy(L->Xb, xb.data(), 2 * n, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (err = cudaMemcpy(L->Tb, host_t, 4 * n, cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_error(err, "fe_lpc_loss_grad: copy");
  double l = 0.0;
  if ((st = mlp_loss_grad(L, batch, 0, &l)) != FE_OK) return st;
  if (host_y && (err = cudaMemcpy(host_y, L->Y, 4 * n, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_error(err, "fe_lpc_loss_grad: y");
  if (host_grad &&
      (err = cudaMemcpy(host_grad, L->grad, 4 * L->nparam, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_error(err, "fe_lpc_loss_grad: grad");
  if (loss) *loss = l;
  return FE_OK;
}

int fe_lpc_adam_step(fe_lpc* L, int batch, const float* host_x, const float* host_t, double lr,
                     double* loss) {
  clear_error();
  if (!L || !host_x || !host_t || batch < 1 || batch > (1 << 20) || !(lr > 0.0))
    return set_error(FE_ERR_ARG, "fe_lpc_adam_step: bad arguments");
  int st = ensure_workspace(L, batch);
  if (st != FE_OK) return st;
  const int64_t n = (int64_t)batch * L->din;
  std::vector<__nv_bfloat16> xb(n);
  for (int64_t i = 0; i < n; ++i) xb[i] = __float2bfloat16(host_x[i]);
  cudaError_t err;
  if ((err = cudaMemcpy(L->Xb, xb.data(), 2 * n, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (err = cudaMemcpy(L->Tb, host_t, 4 * n, cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_error(err, "fe_lpc_adam_step: copy");
  double l = 0.0;
  if ((st = mlp_loss_grad(L, batch, 0, &l)) != FE_OK) return st;
  if ((st = adam_update(L, lr, 0)) != FE_OK) return st;
  if (loss) *loss = l;
  return cuda_error(cudaDeviceSynchronize(), "fe_lpc_adam_step");
}

int fe_lpc_sample_pairs(fe_lpc* L, int reps, int64_t max_rows, int32_t* host_elem,
                        double* host_x, double* host_t, int64_t* rows, void* stream) {
  clear_error();
  if (!L || !rows || max_rows < 0 || (max_rows > 0 && (!host_elem || !host_x || !host_t)))
    return set_error(FE_ERR_ARG, "fe_lpc_sample_pairs: bad arguments");
  if (reps <= 0) reps = 16;
  cudaStream_t s = (cudaStream_t)stream;
  cudaFree(L->Xs);
  cudaFree(L->Ts);
  L->Xs = nullptr;
  L->Ts = nullptr;
  L->nsamp = 0;
  double *xd = nullptr, *td = nullptr;
  std::vector<int32_t> el;
  int st = make_samples(L, reps, s, &xd, &td, &el);
  if (st != FE_OK) return st;
  const int64_t n = max_rows < L->nsamp ? max_rows : L->nsamp;
  cudaError_t err = cudaSuccess;
  if (n > 0) {
    const size_t bytes = sizeof(double) * (size_t)n * L->din;
    if ((err = cudaMemcpyAsync(host_x, xd, bytes, cudaMemcpyDeviceToHost, s)) == cudaSuccess &&
        (err = cudaMemcpyAsync(host_t, td, bytes, cudaMemcpyDeviceToHost, s)) == cudaSuccess)
      err = cudaStreamSynchronize(s);
    for (int64_t r = 0; r < n; ++r) host_elem[r] = el[(size_t)(r / reps)];
  }
  cudaFree(xd);
  cudaFree(td);
  if (err != cudaSuccess) return cuda_error(err, "fe_lpc_sample_pairs: copy");
  *rows = n;
  return FE_OK;
}

int fe_lpc_apply(fe_lpc* L, const double* dev_r, double* dev_z, void* stream) {
  clear_error();
  if (!L || !dev_r || !dev_z) return set_error(FE_ERR_ARG, "fe_lpc_apply: null argument");
  return lpc_apply(L, dev_r, dev_z, (cudaStream_t)stream);
}

int fe_lpc_set_kernel(fe_lpc* L, int kernel) {
  clear_error();
  if (!L) return set_error(FE_ERR_ARG, "fe_lpc_set_kernel: lpc is NULL");
  if (kernel < FE_LPC_KERNEL_AUTO || kernel > FE_LPC_KERNEL_GEMM)
    return set_error(FE_ERR_ARG, "fe_lpc_set_kernel: unknown kernel");
  if (kernel == FE_LPC_KERNEL_TCGEN05 && L->tc_grid <= 0 && L->tc_grid32 <= 0)
    return set_error(FE_ERR_UNSUPPORTED, "fe_lpc_set_kernel: no tcgen05 kernel for this order "
                                         "and width (width 0, 64 or 128 with D^3 <= 128; "
                                         "width 256 with D^3 <= 64)");
  if (kernel == FE_LPC_KERNEL_MMA_SYNC && L->fused_grid <= 0)
    return set_error(FE_ERR_UNSUPPORTED, "fe_lpc_set_kernel: no mma.sync fused kernel for this "
                                         "order and width");
  L->kernel = kernel;
  return FE_OK;
}

int fe_lpc_get_kernel(const fe_lpc* L, int* kernel, int* tc_faults) {
  clear_error();
  if (!L || !kernel) return set_error(FE_ERR_ARG, "fe_lpc_get_kernel: null argument");
  *kernel = lpc_kernel(L, false);
  if (tc_faults) *tc_faults = tc_faulted(L);
  return FE_OK;
}

int fe_lpc_nparams(const fe_lpc* L, int64_t* n) {
  clear_error();
  if (!L || !n) return set_error(FE_ERR_ARG, "fe_lpc_nparams: null argument");
  *n = L->nparam;
  return FE_OK;
}

int fe_fcg(fe_pa* pa, int op, fe_lpc* lpc, const double* dev_b, double* dev_x, double rtol,
           int maxit, fe_pcg_stats* stats, void* stream) {
  clear_error();
  const auto t0 = std::chrono::steady_clock::now();
  if (stats) *stats = fe_pcg_stats{0, 0.0, 0.0, 0.0, 0, 0};
  if (!pa || !dev_b || !dev_x) return set_error(FE_ERR_ARG, "fe_fcg: null argument");
  if (op != FE_DIFFUSION && op != FE_MASS) return set_error(FE_ERR_ARG, "fe_fcg: bad op");
  if (!(pa->ops & op)) return set_error(FE_ERR_ARG, "fe_fcg: operator not set up");
  if (lpc && (lpc->pa != pa || lpc->op != op))
    return set_error(FE_ERR_ARG, "fe_fcg: preconditioner built for another operator");
  if (maxit < 1 || !(rtol >= 0.0)) return set_error(FE_ERR_ARG, "fe_fcg: bad rtol or maxit");
  if (pa->variant == FE_VARIANT_F32)
    return set_error(FE_ERR_UNSUPPORTED, "fe_fcg: the FP32 variant is not FP64-accurate; select "
                                         "FE_VARIANT_F64, F32X2 or F64_DMMA (or use fe_fcg_ir)");
  cudaStream_t s = (cudaStream_t)stream;
  const fe_mesh* m = pa->mesh;
  double* dinv = lpc ? lpc->dinv : nullptr;
  double* own = nullptr;
  int st = FE_OK;
  FcgResult res;
  if (!dinv) {
    cudaError_t err = cudaMalloc(&own, sizeof(double) * m->ndofs);
    if (err != cudaSuccess) return cuda_error(err, "fe_fcg: cudaMalloc");
    dinv = own;
    if ((st = fe_assemble_diagonal(pa, op, dinv, s)) == FE_OK) {
      k_invert_diag<<<grid1(m->ndofs), kT, 0, s>>>(dinv, m->d_mask, m->ndofs);
      res.launches += 2;
    }
  }
  res.stop_at_fallback = lpc && lpc->fallback == FE_PC_CHEBYSHEV;
  if (st == FE_OK) st = fcg_run(pa, op, lpc, dinv, dev_b, dev_x, rtol, maxit, nullptr, s, &res);
  cudaFree(own);
  if (st != FE_OK) return st;
  int cheb_iters = 0;
  if (res.handed_off) {
    // Chebyshev-PCG on the residual equation A d = (1-m)(b - A x) from d = 0, to the tolerance
    // that makes ||b - A (x + d)|| <= rtol ||b||; then x += d.
    const int64_t n = m->ndofs;
    double *buf = nullptr, *red = nullptr;
    cudaError_t err = cudaMalloc(&buf, sizeof(double) * 3 * n);
    if (err == cudaSuccess) err = cudaMalloc(&red, sizeof(double) * (2 * kRB + S_N));
    if (err != cudaSuccess) {
      cudaFree(buf);
      return cuda_error(err, "fe_fcg: fallback workspace");
    }
    double *q = buf, *r = buf + n, *d = buf + 2 * n;
    double hsc[S_N];
    st = apply_dispatch(pa, op, FE_VARIANT_F64, dev_x, q, s);  // FP64 residual
    if (st == FE_OK) {
      cudaMemsetAsync(red + 2 * kRB, 0, sizeof(double) * S_N, s);
      k_ir_resid<<<kRB, kT, 0, s>>>(dev_b, q, m->d_mask, r, n, red, red + kRB);
      k_fcg_finish<<<1, kRB, 0, s>>>(red, red + kRB, red + 2 * kRB, 4);
      res.launches += 3;
      if ((err = cudaGetLastError()) != cudaSuccess ||
          (err = cudaMemcpyAsync(hsc, red + 2 * kRB, sizeof(hsc), cudaMemcpyDeviceToHost, s)) !=
              cudaSuccess ||
          (err = cudaStreamSynchronize(s)) != cudaSuccess)
        st = cuda_error(err, "fe_fcg: fallback residual");
    }
    fe_pcg_stats cs{0, 0.0, 0.0, 0.0, 0, 0};
    int cst = FE_OK;
    if (st == FE_OK) {
      const double rn = sqrt(hsc[S_TRUE]), bn = sqrt(hsc[S_BB]);
      const double rtol_c = rn > 0.0 ? rtol * bn / rn : 1.0;
      cst = fe_pcg_chebyshev(pa, op, 0, 0.0, 0.0, r, d, std::min(rtol_c, 1.0),
                             std::max(1, maxit - res.iters), &cs, stream);
      if (cst == FE_OK || cst == FE_ERR_NOT_CONVERGED) {
        k_add_f64<<<grid1(n), kT, 0, s>>>(dev_x, d, n);
        res.launches += 1 + cs.launches;
        cheb_iters = cs.iters;
        res.rel = bn > 0.0 ? cs.rel_resid * rn / bn : 0.0;
        res.true_rel = bn > 0.0 ? cs.true_rel_resid * rn / bn : 0.0;
        res.status = cst;
        err = cudaStreamSynchronize(s);
        if (err != cudaSuccess) st = cuda_error(err, "fe_fcg: fallback update");
      } else {
        st = cst;
      }
    }
    cudaFree(buf);
    cudaFree(red);
    if (st != FE_OK) return st;
  }
  if (stats) {
    stats->iters = res.iters + cheb_iters;
    stats->rel_resid = res.rel;
    stats->true_rel_resid = res.true_rel;
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    stats->launches = res.launches;
    stats->outer_iters = 1 + res.restarts;
  }
  if (tc_faulted(lpc))
    return set_error(FE_ERR_CUDA, "fe_fcg: the tcgen05 preconditioner gave up a wait on the "
                                  "tensor core");
  switch (res.status) {
    case FE_OK:
      return FE_OK;
    case FE_ERR_BREAKDOWN:
      return set_error(FE_ERR_BREAKDOWN, "fe_fcg: p.Ap <= 0 (operator not SPD on the free dofs)");
    case FE_ERR_NAN:
      return set_error(FE_ERR_NAN, "fe_fcg: NaN or Inf in the iteration");
    default:
      return set_error(FE_ERR_NOT_CONVERGED, "fe_fcg: maxit reached before rtol");
  }
}

// ---- checkpoint: little-endian "FELPC001", int32 din, int32 width, int64 nparam, int32 Adam
// step count, int32 0, then FP32 weights, Adam first and second moments (nparam each).
static const char kLpcMagic[8] = {'F', 'E', 'L', 'P', 'C', '0', '0', '1'};

struct LpcHeader {
  char magic[8];
  int32_t din, width;
  int64_t nparam;
  int32_t adam_t, pad;
};
static_assert(sizeof(LpcHeader) == 32, "checkpoint header layout");

static int read_lpc_header(FILE* f, LpcHeader* h, const char* who) {
  if (std::fread(h, sizeof(*h), 1, f) != 1 || std::memcmp(h->magic, kLpcMagic, 8) != 0)
    return set_error(FE_ERR_ARG, std::string(who) + ": not a preconditioner checkpoint");
  if (h->din < 1 || h->width < 0 || h->nparam < 1 || h->adam_t < 0)
    return set_error(FE_ERR_ARG, std::string(who) + ": corrupt checkpoint header");
  return FE_OK;
}

int fe_lpc_checkpoint_info(const char* path, int* din, int* width, int64_t* nparam,
                           int* adam_steps) {
  clear_error();
  if (!path) return set_error(FE_ERR_ARG, "fe_lpc_checkpoint_info: path is NULL");
  FILE* f = std::fopen(path, "rb");
  if (!f) return set_error(FE_ERR_ARG, std::string("fe_lpc_checkpoint_info: cannot open ") + path);
  LpcHeader h;
  const int st = read_lpc_header(f, &h, "fe_lpc_checkpoint_info");
  std::fclose(f);
  if (st != FE_OK) return st;
  if (din) *din = h.din;
  if (width) *width = h.width;
  if (nparam) *nparam = h.nparam;
  if (adam_steps) *adam_steps = h.adam_t;
  return FE_OK;
}

int fe_lpc_save(fe_lpc* L, const char* path) {
  clear_error();
  if (!L || !path) return set_error(FE_ERR_ARG, "fe_lpc_save: null argument");
  const int64_t n = L->nparam;
  std::vector<float> w(n), m(n, 0.0f), v(n, 0.0f);
  cudaError_t err = cudaMemcpy(w.data(), L->w32, 4 * n, cudaMemcpyDeviceToHost);
  if (err == cudaSuccess) err = cudaMemcpy(m.data(), L->adam_m, 4 * n, cudaMemcpyDeviceToHost);
  if (err == cudaSuccess) err = cudaMemcpy(v.data(), L->adam_v, 4 * n, cudaMemcpyDeviceToHost);
  if (err != cudaSuccess) return cuda_error(err, "fe_lpc_save: copy");
  LpcHeader h;
  std::memcpy(h.magic, kLpcMagic, 8);
  h.din = L->din;
  h.width = L->width;
  h.nparam = n;
  h.adam_t = L->adam_t;
  h.pad = 0;
  FILE* f = std::fopen(path, "wb");
  if (!f) return set_error(FE_ERR_ARG, std::string("fe_lpc_save: cannot open ") + path);
  const bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1 &&
                  std::fwrite(w.data(), 4, n, f) == (size_t)n &&
                  std::fwrite(m.data(), 4, n, f) == (size_t)n &&
                  std::fwrite(v.data(), 4, n, f) == (size_t)n;
  if (std::fclose(f) != 0 || !ok) return set_error(FE_ERR_ARG, "fe_lpc_save: write failed");
  return FE_OK;
}

int fe_lpc_load(fe_lpc* L, const char* path) {
  clear_error();
  if (!L || !path) return set_error(FE_ERR_ARG, "fe_lpc_load: null argument");
  FILE* f = std::fopen(path, "rb");
  if (!f) return set_error(FE_ERR_ARG, std::string("fe_lpc_load: cannot open ") + path);
  LpcHeader h;
  int st = read_lpc_header(f, &h, "fe_lpc_load");
  if (st == FE_OK && (h.din != L->din || h.width != L->width || h.nparam != L->nparam))
    st = set_error(FE_ERR_ARG, "fe_lpc_load: checkpoint of another network shape");
  const int64_t n = L->nparam;
  std::vector<float> w, m, v;
  if (st == FE_OK) {
    w.resize(n);
    m.resize(n);
    v.resize(n);
    if (std::fread(w.data(), 4, n, f) != (size_t)n || std::fread(m.data(), 4, n, f) != (size_t)n ||
        std::fread(v.data(), 4, n, f) != (size_t)n)
      st = set_error(FE_ERR_ARG, "fe_lpc_load: truncated checkpoint");
  }
  std::fclose(f);
  if (st != FE_OK) return st;
  cudaError_t err = cudaMemcpy(L->w32, w.data(), 4 * n, cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemcpy(L->adam_m, m.data(), 4 * n, cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemcpy(L->adam_v, v.data(), 4 * n, cudaMemcpyHostToDevice);
  if (err != cudaSuccess) return cuda_error(err, "fe_lpc_load: copy");
  L->adam_t = h.adam_t;
  k_to_bf16<<<grid1(n), kT>>>(L->w32, L->wb, n);
  L->wimg_ok = false;
  L->tcimg_ok = false;
  return cuda_error(cudaDeviceSynchronize(), "fe_lpc_load");
}

int fe_pa_set_learned(fe_pa* pa, fe_lpc* lpc) {
  clear_error();
  if (!pa) return set_error(FE_ERR_ARG, "fe_pa_set_learned: pa is NULL");
  if (lpc && lpc->pa != pa)
    return set_error(FE_ERR_ARG, "fe_pa_set_learned: preconditioner built for another fe_pa");
  pa->lpc = lpc;
  return FE_OK;
}

int fe_lpc_set_fallback(fe_lpc* lpc, int pc) {
  clear_error();
  if (!lpc) return set_error(FE_ERR_ARG, "fe_lpc_set_fallback: lpc is NULL");
  if (pc != FE_PC_JACOBI && pc != FE_PC_CHEBYSHEV)
    return set_error(FE_ERR_ARG, "fe_lpc_set_fallback: pc must be FE_PC_JACOBI or FE_PC_CHEBYSHEV");
  lpc->fallback = pc;
  return FE_OK;
}

void fe_lpc_destroy(fe_lpc* L) {
  if (!L) return;
  if (L->pa && L->pa->lpc == L) L->pa->lpc = nullptr;
  cudaFree(L->w32); cudaFree(L->wb); cudaFree(L->adam_m); cudaFree(L->adam_v); cudaFree(L->grad);
  cudaFree(L->wsq); cudaFree(L->dinv); cudaFree(L->dis); cudaFree(L->fsc); cudaFree(L->fsc32); cudaFree(L->wimg); cudaFree(L->tcimg); cudaFree(L->d_tcfail); cudaFree(L->red); cudaFree(L->Xs); cudaFree(L->Ts);
  cudaFree(L->Xb); cudaFree(L->H1b); cudaFree(L->H2b); cudaFree(L->dYb); cudaFree(L->dA1b);
  cudaFree(L->dA2b); cudaFree(L->Z1); cudaFree(L->Z2); cudaFree(L->Y); cudaFree(L->Tb);
  cudaFree(L->scale);
  delete L;
}

}  // extern "C"
