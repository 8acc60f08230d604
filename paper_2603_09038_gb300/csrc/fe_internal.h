// Internal declarations of libfe (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <string>

#include "../../include/fe.h"

namespace fe {

constexpr int kMaxOrder = 8;
// built launch shapes of the fused apply per arithmetic (fe_apply_launch.cuh lists them)
constexpr int kShapesF64 = 3, kShapesF32x2 = 3;
constexpr int kMaxD = kMaxOrder + 1;
constexpr int kMaxQ = kMaxOrder + 2;

// Records msg as the calling thread's last error and returns status.
int set_error(int status, const std::string& msg);
int cuda_error(cudaError_t err, const char* what);
void clear_error();

// 1D tables for order p with a q-point Gauss rule on [0, 1] (host, FP64):
// nodes[d] GLL nodes, pts[q]/wts[q] Gauss-Legendre rule, B[q*D+d] = l_d(x_q), G[q*D+d] = l_d'(x_q).
struct Basis1D {
  int p = 0, D = 0, Q = 0;
  double nodes[kMaxD];
  double pts[kMaxQ];
  double wts[kMaxQ];
  double B[kMaxQ * kMaxD];
  double G[kMaxQ * kMaxD];
};
// Returns false if p or q is out of range.
bool make_basis_1d(int p, int q, Basis1D* out);
// Lagrange basis of the p+1 Gauss-Legendre points of [0, 1] (a discontinuous L2 basis) at the
// q-point Gauss-Legendre rule: Bl[i*(p+1) + d] = l_d(x_i).  False if out of range.
bool make_l2_basis_1d(int p, int q, double* Bl);

// y = A x with the FP32 variant on float vectors (the caller zeroes y); same skip / dot_part
// semantics as apply_dispatch.
int apply_f32_vectors(const fe_pa* pa, int op, const float* x, float* y, cudaStream_t s,
                      const int* skip, double* dot_part);

// Learned patch preconditioner hooks of the variable-order space (fe_learned.cu): z (+)= M(r) on
// the handle's mesh numbering; shape; weight copy; external input/output scaling.
int lpc_apply(fe_lpc* L, const double* r, double* z, cudaStream_t s, bool accumulate);
void lpc_shape(const fe_lpc* L, int* order, int* din, int* width);
int lpc_copy_weights(fe_lpc* dst, const fe_lpc* src, cudaStream_t s);
int lpc_set_scaling(fe_lpc* L, const double* F, cudaStream_t s);

// Flexible CG (fe_learned.cu) on an arbitrary FP64 operator of n dofs with boundary mask `mask`:
// apply (out = A in), prec (z = M(r), the learned preconditioner; FCG falls back to Jacobi with
// dinv when it stalls), true_apply (the FP64 operator for the exit true residual).  Fills
// *stats; returns the solver status (FE_OK, FE_ERR_NOT_CONVERGED, FE_ERR_BREAKDOWN, FE_ERR_NAN)
// or an error.  Synchronous.
struct FcgOperator {
  int64_t n = 0;
  const uint8_t* mask = nullptr;
  std::function<int(const double*, double*)> apply, prec, true_apply;
};
int fcg_solve(const FcgOperator& op, const double* dinv, const double* b, double* x, double rtol,
              int maxit, cudaStream_t s, fe_pcg_stats* stats, const char* who);

}  // namespace fe

struct fe_mesh {
  int nx = 0, ny = 0, nz = 0, p = 0, D = 0;
  int64_t ne = 0, ndofs = 0;
  int64_t Nx = 0, Ny = 0, Nz = 0;  // GLL lattice points per axis
  int device = 0;
  double* d_vertices = nullptr;    // [(nx+1)(ny+1)(nz+1)][3]
  int32_t* d_map = nullptr;        // [ne][D^3]
  uint8_t* d_mask = nullptr;       // [ndofs]
  // An element subset of an nx x ny x nz mesh (the order groups of a variable-order space):
  // mesh index of every element, NULL for the whole structured mesh.
  int32_t* d_elem_ids = nullptr;
};

struct fe_pa {
  const fe_mesh* mesh = nullptr;   // not owned; must outlive the fe_pa
  int p = 0, D = 0, Q = 0, ops = 0;
  int variant = FE_VARIANT_F64;
  fe::Basis1D basis;
  // FP64 quadrature data, always kept (FE_VARIANT_F64, DMMA, the diagonal and every FP64
  // residual of the solvers read it)
  double* d_qd_diff = nullptr;     // [ne][Q][6][Q][Q] (qz, component, qy, qx)
  double* d_qd_mass = nullptr;     // [ne][Q][Q][Q]
  double* d_coeff = nullptr;       // [ne] copy of the coefficient (nullptr => 1)
  // FE_VARIANT_F32X2 copy (made on first use): per element e, the entries times 2^-s_e as
  // (hi, lo) float pairs in the same layout, s_e in d_qs_* (the element's largest entry times
  // 2^-s_e lies in [1, 2))
  double* d_qd_diff2 = nullptr;
  double* d_qd_mass2 = nullptr;
  int32_t* d_qs_diff = nullptr;    // [ne]
  int32_t* d_qs_mass = nullptr;    // [ne]
  float* d_qd_diff32 = nullptr;    // FP32 copy for FE_VARIANT_F32 (made on first use), times
  float* d_qd_mass32 = nullptr;    // 2^-qd32_shift[op] (its largest entry in [1, 2))
  int qd32_shift[2] = {0, 0};      // diffusion, mass
  int shape[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};  // launch shape per (operator, variant)
  // PCG workspace (allocated on first fe_pcg, freed by fe_pa_destroy)
  double* d_work = nullptr;        // 5 vectors of ndofs
  double* d_red = nullptr;         // reduction partials + scalars
  int* d_flags = nullptr;
  int64_t work_ndofs = 0;
  double* d_dpart = nullptr;       // per-block partials of the apply-fused p.Ap
  double* d_hostio = nullptr;      // device b and x of fe_pcg_host (2 vectors of ndofs)
  int64_t dpart_cap = 0;
  double cheb_lmax[2] = {0.0, 0.0};  // cached lambda_max estimates of D^-1 A (diffusion, mass)
  bool pcg_graphs = true;          // fe_pcg replays its iteration batches as CUDA graphs
  fe_lpc* lpc = nullptr;           // learned preconditioner for FE_PC_LEARNED (not owned)
};

namespace fe {

// Arguments of one apply launch.
struct ApplyArgs {
  const int32_t* map;
  const double* qd;      // FP64 or float-pair encoded, per variant
  const int32_t* qscale = nullptr;  // per-element scale exponents of float-pair data
  int qshift = 0;        // FP32 data: results on FP64 vectors are scaled by 2^qshift
  const double* x;
  double* y;
  int64_t ne;
  int p, Q;
  const Basis1D* basis;
  const int* skip;       // optional device flag; nonzero => the launch does nothing
  double* dot_part;      // optional: per-block partials of sum_e x_e . (A_e x_e) (= x^T A x)
  int64_t* blocks;       // optional out: grid size of the launch (set also when query_only)
  bool query_only;       // only report the grid size
  int nrhs = 1;          // right-hand sides x + r ldx -> y + r ldy, r < nrhs
  int64_t ldx = 0, ldy = 0;
  int shape = 0;         // launch shape index (fe_pa_set_shape)
  int* elems_per_block = nullptr;    // optional outs: the launch shape's geometry
  int* threads_per_block = nullptr;
};

// Order groups of a variable-order space for the persistent multi-order apply: group i has
// elements of order order[i] (an element list with its own dof-map slice, quadrature data and,
// for float pairs, scales); its work items are first_item[i] .. first_item[i + 1] - 1, each a
// block of multi_elems(variant, op, order) consecutive elements of the list.
struct MultiGroups {
  int n = 0;
  int order[kMaxOrder];
  int64_t first_item[kMaxOrder + 1];
  const int32_t* map[kMaxOrder];
  const double* qd[kMaxOrder];
  const int32_t* qscale[kMaxOrder];
  int64_t ne[kMaxOrder];
};
// Elements per work item of the multi-order apply (FE_VARIANT_F64 or FE_VARIANT_F32X2), 0 if not
// built; one persistent launch over the groups (y zeroed by the caller; counter: a device int).
int multi_elems(int variant, int op, int order);
int launch_apply_multi(int variant, int op, const MultiGroups& g, const Basis1D* const* basis,
                       const double* x, double* y, int* counter, int nrhs, int64_t ldx,
                       int64_t ldy, cudaStream_t s);

// A linear operator for the batched CG (fe_pcg_batched, fe_vspace_pcg_batched): n unknowns,
// the boundary mask (essential dofs), Q_j = A P_j for nr search directions stored with leading
// dimension n (skip: a device flag the kernels may test to do nothing once every system has
// stopped; Q is zeroed beforehand), the same with the FP64 operator for the true residuals
// (X with leading dimension lx), and the Jacobi diagonal (empty: no preconditioner).  nk counts
// the kernels launched.  graphs: replay iteration batches as CUDA graphs.
struct BatchedOperator {
  int64_t n = 0;
  const uint8_t* mask = nullptr;
  std::function<int(cudaStream_t, int, const double*, double*, const int*, int*)> apply;
  std::function<int(cudaStream_t, int, const double*, int64_t, double*, int*)> apply_fp64;
  std::function<int(cudaStream_t, double*)> diagonal;
  bool graphs = true;
};
int pcg_batched_core(const BatchedOperator& A, int nrhs, const double* dev_b, int64_t ldb,
                     double* dev_x, int64_t ldx, double rtol, int maxit, fe_pcg_stats* stats,
                     cudaStream_t s, const char* who);

// Launchers (one translation unit per variant); return FE_OK or an error status.
int launch_apply_f64(int op, const ApplyArgs& a, cudaStream_t s);
int launch_apply_f32x2(int op, const ApplyArgs& a, cudaStream_t s);
int launch_apply_dmma(int op, const ApplyArgs& a, cudaStream_t s);
int launch_apply_f32(int op, const ApplyArgs& a, cudaStream_t s);
int launch_apply_f32_vec32(int op, const ApplyArgs& a, cudaStream_t s);
// FP32 copy of n FP64 quadrature values times 2^-*shift, *shift chosen so that the largest
// lies in [1, 2) (the copy then spans the float range whatever the coefficient's magnitude).
int make_qd_f32(const double* src, float* dst, int64_t n, int* shift, cudaStream_t s);
int multi_elems_f64(int op, int order);
int multi_elems_f32x2(int op, int order);
int launch_apply_multi_f64(int op, const MultiGroups& g, const Basis1D* const* basis,
                           const double* x, double* y, int* counter, int nrhs, int64_t ldx,
                           int64_t ldy, cudaStream_t s);
int launch_apply_multi_f32x2(int op, const MultiGroups& g, const Basis1D* const* basis,
                             const double* x, double* y, int* counter, int nrhs, int64_t ldx,
                             int64_t ldy, cudaStream_t s);

// diag += the element diagonals of op scattered through the element map (no zeroing; atomic).
int diagonal_accumulate(const fe_pa* pa, int op, double* diag, cudaStream_t s);

// Float-pair copy of FP64 quadrature data: per element (per_elem values each) the scale
// exponent s_e of its largest entry and the entries times 2^-s_e as (hi, lo) pairs.
int encode_f32x2(const double* src, double* dst, int32_t* scale, int64_t ne, int per_elem,
                 cudaStream_t s);

// y = A x (y zeroed first unless skip is given; with skip the caller zeroes y).  skip:
// optional device flag, nonzero => no-op.  dot_part: optional per-block partials of x^T A x
// (variants F64, F32X2, F32); blocks: optional out, the grid size (number of partials).
int apply_dispatch(const fe_pa* pa, int op, int variant, const double* x, double* y,
                   cudaStream_t s, const int* skip = nullptr, double* dot_part = nullptr,
                   int64_t* blocks = nullptr, bool query_only = false, int nrhs = 1,
                   int64_t ldx = 0, int64_t ldy = 0, int* elems_per_block = nullptr,
                   int* threads_per_block = nullptr);
// Number of built launch shapes of a variant (FE_VARIANT_F64_DMMA: 1).
int apply_shape_count(int variant);

// y = A x with the FP32 variant on float vectors (the caller zeroes y); same skip / dot_part
// semantics as apply_dispatch.
int apply_f32_vectors(const fe_pa* pa, int op, const float* x, float* y, cudaStream_t s,
                      const int* skip, double* dot_part);

}  // namespace fe
