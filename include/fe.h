/*
 * fe.h -- C ABI of libfe: GB300-native partial-assembly (PA) finite element operators.
 *
 * The library applies the high-order H1 diffusion and mass operators on hexahedral meshes in the
 * matrix-free partial-assembly form  y = P^T G^T B^T D B G P x  (paper Section II-B, Eq. (1)):
 *   G   element restriction (gather of element dofs through a dof map; G^T is scatter-add),
 *   B   tensor-product basis, applied by sum factorisation as 1D contractions (Eq. (2)),
 *   D   the block-diagonal operator at quadrature points, precomputed once ("partial assembly"),
 *   P   the parallel restriction, the identity on one GPU.
 * Each apply is one fused CUDA kernel: gather, forward contractions, D, transposed
 * contractions and atomic scatter-add (the fusion of Section III-G).
 *
 * Conventions (every entry point):
 *  - Returns FE_OK (0) or a negative fe_status; nothing aborts, traps or asserts on the device.
 *    fe_last_error() gives a message for the calling thread's last non-OK status.
 *  - "dev_" pointers are caller-owned device memory (e.g. torch.empty(..., device='cuda')
 *    .data_ptr()); "host_" pointers are caller-owned host memory.  Vectors are FP64, length
 *    ndofs, contiguous.  Input and output vectors must not alias.
 *  - "stream" is a cudaStream_t passed as void* (NULL = the legacy default stream).  Applies are
 *    asynchronous and stream-ordered; setup calls and fe_pcg synchronise the stream.
 *  - Handles (fe_mesh, fe_pa) are opaque, library-owned, freed by their *_destroy function, and
 *    not safe for concurrent use from several host threads.
 *
 * Numbering (the paper is silent; standard lexicographic choices): elements e = ex + nx*(ey +
 * ny*ez); element-local dofs a = i + D*(j + D*k), D = order+1 (x fastest); global dofs on the
 * (nx*p+1)(ny*p+1)(nz*p+1) GLL lattice, x fastest; vertices on the (nx+1)(ny+1)(nz+1) lattice.
 */
#ifndef FE_H
#define FE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fe_mesh fe_mesh;
typedef struct fe_pa fe_pa;

typedef enum {
  FE_OK = 0,
  FE_ERR_ARG = -1,           /* invalid argument (null pointer, bad size, inverted element, ...) */
  FE_ERR_CUDA = -2,          /* a CUDA runtime call failed; see fe_last_error()                  */
  FE_ERR_OOM = -3,           /* device allocation failed                                         */
  FE_ERR_UNSUPPORTED = -4,   /* order / quadrature / variant combination not built               */
  FE_ERR_NOT_CONVERGED = -5, /* fe_pcg hit maxit before reaching rtol                            */
  FE_ERR_BREAKDOWN = -6,     /* fe_pcg found p.Ap <= 0 (operator not SPD on the free dofs)        */
  FE_ERR_NAN = -7,           /* fe_pcg met a NaN or Inf                                          */
  FE_ERR_TIMEOUT = -8        /* reserved for a bounded device-side wait that ran out; no entry
                                point returns it (no kernel of the library waits on another)    */
} fe_status;

typedef enum { FE_DIFFUSION = 1, FE_MASS = 2 } fe_op;

/* FE_PC_LEARNED: flexible CG with the learned preconditioner attached by fe_pa_set_learned
 * (fe_pcg only; it is fe_fcg with that preconditioner). */
typedef enum { FE_PC_NONE = 0, FE_PC_JACOBI = 1, FE_PC_CHEBYSHEV = 2, FE_PC_LEARNED = 3 } fe_pc;

/* Arithmetic of the apply kernels.  All variants take and return FP64 vectors.
 *  FE_VARIANT_F64     FP64 FMA on the FP64 pipe (IEEE double throughout).
 *  FE_VARIANT_F32X2   FP64-accurate float-float ("double-FP32") arithmetic on the FP32 pipe:
 *                     each value is an unevaluated sum hi + lo of two floats (about 47 bits of
 *                     significand), products and sums by error-free transformations (Dekker's
 *                     product with FMA, Knuth's TwoSum).  Power-of-two scales make it cover the
 *                     whole FP64 range: each thread block's gathered inputs are scaled so that
 *                     the largest lies in [1, 2), each element's quadrature data likewise (the
 *                     scale is stored with the float-pair copy), and both scales are undone when
 *                     the results are widened to FP64.  Inputs below 2^-126 times the largest
 *                     input of their block, and FP64 subnormals, count as zero (relative effect
 *                     below 1e-38 of the block's scale).
 *  FE_VARIANT_F64_DMMA FP64 with the 1D contractions on the FP64 tensor-core instruction
 *                     mma.sync.m8n8k4.f64 (the paper's DMMA, Section III-B).
 *  FE_VARIANT_F32     plain FP32 arithmetic on an FP32 copy of the quadrature data (made on
 *                     first use): NOT FP64-accurate (relative error ~1e-6); it is the inner
 *                     operator of fe_pcg_ir's mixed-precision iterative refinement.          */
typedef enum {
  FE_VARIANT_F64 = 0,
  FE_VARIANT_F32X2 = 1,
  FE_VARIANT_F64_DMMA = 2,
  FE_VARIANT_F32 = 3
} fe_variant;

typedef struct {
  int iters;             /* iterations performed                                              */
  double rel_resid;      /* recursive ||r||_2 / ||b||_2 at exit                               */
  double true_rel_resid; /* ||b - A x||_2 / ||b||_2 recomputed at exit with FE_VARIANT_F64 (FP64
                            quadrature data and FP64 arithmetic), whatever variant iterated */
  double seconds;        /* host wall time of the call, including the diagonal assembly       */
  int launches;          /* kernels of this library launched by the call (no-op ones included) */
  int outer_iters;       /* refinement steps (fe_pcg_ir); 1 for fe_pcg                        */
} fe_pcg_stats;

/* Builds the mesh topology on the device: the element dof map (int32 [ne][D^3], the G of
 * Eq. (1)), the boundary-dof mask and the 1D GLL nodes.  host_vertices: FP64
 * [(nx+1)(ny+1)(nz+1)][3], x fastest, copied.  order 1..8.  Synchronous. */
int fe_mesh_setup(int nx, int ny, int nz, int order, const double* host_vertices, fe_mesh** out);

/* The 1D tables of Eq. (2) that every apply uses (host only, no device needed): nodes[D] the
 * order+1 Gauss-Lobatto-Legendre nodes on [0,1], pts[Q] / wts[Q] the q1d-point Gauss-Legendre
 * rule on [0,1], B[Q][D] = l_d(x_q) and G[Q][D] = l_d'(x_q) (row-major, q slowest), computed in
 * long double and rounded once.  Any output may be NULL.  FE_ERR_ARG unless order is 1..8 and
 * q1d 1..10. */
int fe_basis_1d(int order, int q1d, double* nodes, double* pts, double* wts, double* B,
                double* G);

/* Sizes of a mesh: global dofs (incl. boundary; the L-vector length of Eq. (1)), elements,
 * order. */
int fe_mesh_sizes(const fe_mesh* mesh, int64_t* ndofs, int64_t* nelems, int* order);

/* Global dofs of a mesh (incl. boundary); the first output of fe_mesh_sizes. */
int fe_mesh_ndofs(const fe_mesh* mesh, int64_t* ndofs);

/* Copies the boundary-dof mask (uint8 [ndofs], 1 on the cube's boundary lattice) to dev_mask:
 * the essential-condition set of the solvers (the paper is silent; homogeneous Dirichlet). */
int fe_mesh_boundary_mask(const fe_mesh* mesh, uint8_t* dev_mask, void* stream);

/* Copies the element dof map (int32 [ne][D^3]) to dev_map: the index gather of G in Eq. (1),
 * the indirect reads of Section III-G. */
int fe_mesh_dof_map(const fe_mesh* mesh, int32_t* dev_map, void* stream);

/* Partial assembly (Section II-B: the block-diagonal D at the quadrature points is evaluated once
 * and kept).  Computes per element and Gauss point the trilinear Jacobian J, det J and
 * adj(J), and stores
 *   diffusion  D_q = w_q c_e adj(J) adj(J)^T / det J   (6 symmetric entries)
 *   mass       M_q = w_q c_e det J
 * q1d: Gauss points per axis, 0 => order+2 (the only value built).  dev_coeff: FP64 [ne]
 * piecewise-constant coefficient, or NULL for 1.  ops: FE_DIFFUSION | FE_MASS (bitwise or).
 * Fails with FE_ERR_ARG if an element has det J <= 0 at a Gauss point.  Synchronous. */
int fe_pa_setup(const fe_mesh* mesh, int q1d, const double* dev_coeff, int ops, void* stream,
                fe_pa** out);

/* Selects the arithmetic of subsequent applies (Sections III-B/F: FMA or DMMA; float-float and
 * FP32 are extensions).  The FP64 quadrature data are always kept (the FP64 residuals of the
 * solvers and the diagonal read them); the first selection of FE_VARIANT_F32X2 adds a
 * float-pair copy (same size, plus one int32 scale exponent per element), the first selection
 * of FE_VARIANT_F32 an FP32 copy (half the size, shifted by a power of two into the float
 * range); both are kept until fe_pa_destroy.  Synchronous when a copy is made. */
int fe_pa_set_variant(fe_pa* pa, int variant, void* stream);
int fe_pa_get_variant(const fe_pa* pa, int* variant);

/* Launch shape of the fused apply for (op, variant): every arithmetic has a few built shapes
 * (threads per block, and a shared-memory budget that fixes the elements per block: shape 0 the
 * default for most orders, others with smaller blocks and more of them per SM; the float-float
 * default is the smaller-block shape 1 where it measured faster: diffusion p <= 2, mass p <= 4
 * and p = 8).  fe_pa_set_shape selects one
 * (FE_ERR_ARG if the index is not built for the variant); fe_pa_get_shape returns the selected
 * index, the number of built shapes, and the threads and elements per block of the selected
 * shape for this handle's order (0 for FE_VARIANT_F64_DMMA, whose kernel has one fixed shape);
 * any output may be NULL. */
int fe_pa_set_shape(fe_pa* pa, int op, int variant, int shape);
int fe_pa_get_shape(const fe_pa* pa, int op, int variant, int* shape, int* nshapes,
                    int* threads_per_block, int* elems_per_block);

/* Autotuner of the arithmetic and the launch shape (an extension): times one apply of op (nrhs
 * right-hand sides in one batched launch, 1..64) with each FP64-accurate variant --
 * FE_VARIANT_F32X2, FE_VARIANT_F64 and, for nrhs = 1, FE_VARIANT_F64_DMMA -- in each of its
 * built launch shapes, as the mean of `reps` launches after one warm-up (CUDA events on
 * `stream`); keeps the fastest shape of every variant (fe_pa_get_shape reports it), selects the
 * fastest variant with fe_pa_set_variant and returns it in *best_variant; ms (NULL or double[4],
 * indexed by fe_variant) gets each variant's time in its fastest shape, -1 where not timed.
 * FE_VARIANT_F32 is not a candidate (not FP64-accurate).  Allocates 2 nrhs vectors of scratch.
 * Synchronous. */
int fe_pa_autotune(fe_pa* pa, int op, int nrhs, int reps, int* best_variant, double* ms,
                   void* stream);

/* y = A x = G^T B^T D B G x on the full L-vector (Eq. (1) with P the identity; B by sum
 * factorisation, Eq. (2); one fused kernel, Section III-G), no boundary conditions, with the
 * handle's variant.
 * Overwrites y (it is zeroed, then accumulated by atomic scatter-add).  Asynchronous. */
int fe_apply_diffusion(const fe_pa* pa, const double* dev_x, double* dev_y, void* stream);
int fe_apply_mass(const fe_pa* pa, const double* dev_x, double* dev_y, void* stream);
/* Same for op = FE_DIFFUSION or FE_MASS with an explicit variant. */
int fe_apply(const fe_pa* pa, int op, int variant, const double* dev_x, double* dev_y,
             void* stream);

/* Batched apply (an extension beyond the paper: many right-hand sides per launch): y_r = A x_r for
 * r < nrhs, x_r = dev_x + r*ldx, y_r = dev_y + r*ldy (leading dimensions in elements, >= ndofs).
 * One launch; every thread block applies all right-hand sides to its elements one after the
 * other, so after the first one its dof map and quadrature data are read from L2 instead of
 * HBM.  Variants F64, F32X2 and F32 (not DMMA).  y is zeroed first.  Asynchronous. */
int fe_apply_batched(const fe_pa* pa, int op, int variant, int nrhs, const double* dev_x,
                     int64_t ldx, double* dev_y, int64_t ldy, void* stream);

/* diag(A) of Eq. (1)'s operator (the Jacobi diagonal; the paper is silent on solvers), no
 * boundary conditions, by a sum-factorised diagonal kernel in FP64 (with
 * FE_VARIANT_F32X2 data, each stored pair is widened to FP64 first).  Asynchronous. */
int fe_assemble_diagonal(const fe_pa* pa, int op, double* dev_diag, void* stream);

/* Test problem (the paper is silent): load vector of -div grad u = f, u = sin(pi x) sin(pi y)
 * sin(pi z):
 * b_a = sum_e sum_q w_q det J f(x_q) phi_a(x_q), f = 3 pi^2 u, with the operator's Gauss rule.
 * Asynchronous. */
int fe_load_vector_sine(const fe_pa* pa, double* dev_b, void* stream);

/* The solver around Eq. (1)'s operator (the paper is silent; the time-to-solution metric):
 * Jacobi- (or un-, or Chebyshev-, or learned-) preconditioned CG for A_bc x = b with homogeneous
 * Dirichlet conditions on the mesh boundary: A_bc = (1-m) A (1-m) + m (m = boundary mask).  b's boundary entries are
 * ignored; x is overwritten (zero initial guess; x = 0 on the boundary).  Stops when the
 * recursive residual satisfies ||r||_2 <= rtol ||b||_2 or after maxit iterations.  FP64 vectors
 * and deterministic FP64 inner products (p.Ap included, accumulated in FP64 inside the fused
 * apply from the FP64 results it scatters); applies use the handle's variant, which must be
 * FP64-accurate (FE_ERR_UNSUPPORTED for FE_VARIANT_F32); the exit true residual uses the FP64
 * operator.  Work vectors are allocated on first use and cached in the handle.  Synchronous;
 * fills *stats (may be NULL).  Returns FE_OK, FE_ERR_NOT_CONVERGED, FE_ERR_BREAKDOWN or
 * FE_ERR_NAN (x holds the last iterate in every case). */
int fe_pcg(fe_pa* pa, int op, int pc, const double* dev_b, double* dev_x, double rtol, int maxit,
           fe_pcg_stats* stats, void* stream);

/* fe_pcg through host buffers: the call an application makes with its vectors in host memory.
 * host_b [ndofs] is copied to the device on `stream`, the system is solved as by fe_pcg (same
 * op, pc, rtol, maxit and statuses), and the solution is copied back into host_x [ndofs].  Both
 * arrays are caller-owned host memory; page-locked (pinned) arrays make the two copies DMA
 * transfers, pageable ones work too (the driver stages them).  The device copies of b and x are
 * allocated on first use and cached in the handle (freed by fe_pa_destroy).  host_x receives
 * the last iterate whenever the solve ran (FE_OK, FE_ERR_NOT_CONVERGED, FE_ERR_BREAKDOWN,
 * FE_ERR_NAN); on FE_ERR_ARG, FE_ERR_UNSUPPORTED, FE_ERR_OOM or a failed copy (FE_ERR_CUDA) it is
 * left untouched.  Synchronous; stats->seconds includes both copies. */
int fe_pcg_host(fe_pa* pa, int op, int pc, const double* host_b, double* host_x, double rtol,
                int maxit, fe_pcg_stats* stats, void* stream);

/* PCG with a Chebyshev polynomial preconditioner (an extension; the paper uses no solver here):
 * z = q(D^-1 A_bc) D^-1 r from `degree` steps of the Chebyshev semi-iteration for
 * D^-1 A_bc z = D^-1 r, started at z = 0, on the interval [hi / lmin_ratio, hi], so that
 * 1 - lam q(lam) = T_degree((theta - lam) / delta) / T_degree(theta / delta) (theta, delta the
 * interval's centre and half-width, T the Chebyshev polynomial).  q is positive on (0, hi], so
 * the preconditioner is linear and SPD when hi bounds the spectrum of D^-1 A_bc.  Each iteration
 * costs `degree` applies (one for CG, degree - 1 for the polynomial).
 *   degree      1..32, 0 => 4 (degree 1 is Jacobi scaled by 1/theta);
 *   lmax        hi; 0 => 1.1 x fe_estimate_lmax with 20 power steps, computed on the first such
 *               call for this handle and operator and cached in the handle;
 *   lmin_ratio  hi / lo > 1; 0 => 30.
 * Everything else (system, stopping rule, stats, status codes) as fe_pcg; fe_pcg with
 * pc = FE_PC_CHEBYSHEV calls this with the defaults.  Work vectors: 7 of ndofs, cached. */
int fe_pcg_chebyshev(fe_pa* pa, int op, int degree, double lmax, double lmin_ratio,
                     const double* dev_b, double* dev_x, double rtol, int maxit,
                     fe_pcg_stats* stats, void* stream);

/* Largest-eigenvalue estimate of D^-1 A_bc for the Chebyshev preconditioner (an extension;
 * D = diag(A), boundary rows and columns removed):
 * `iters` power steps (0..1000) from a fixed pseudo-random start, then the generalised Rayleigh
 * quotient (v.Av)/(v.Dv) of the last iterate, a lower bound of lambda_max.  Synchronous. */
int fe_estimate_lmax(fe_pa* pa, int op, int iters, double* lmax, void* stream);

/* CUDA-graph replay of fe_pcg's iterations (an extension).  fe_pcg (Jacobi / none) enqueues its
 * iterations in batches of 8 between two reads of the
 * device-resident stop flag.  By default the first batch is launched kernel by kernel and the
 * next ones are one captured CUDA graph of 8 iterations replayed with a single launch each
 * (captured on a private stream, so any caller stream works; if the capture fails, the kernels
 * are launched one by one).  enable = 0 turns the graphs off for this handle (same kernels and
 * results, more launch overhead on small meshes). */
int fe_pcg_set_graphs(fe_pa* pa, int enable);

/* Mixed-precision iterative refinement around an FP32 inner PCG (an extension; the paper
 * itself stays in FP64 throughout).  Outer loop, in FP64 vectors:
 *   r = (1-m)(b - A x)   with the FP64 operator (FE_VARIANT_F64: FP64 data and arithmetic);
 *   solve A_bc d = r     by PCG (pc) with the FE_VARIANT_F32 operator to inner_rtol * ||r||
 *                        (0 => 1e-2, the fastest setting measured on the 64^3 p=3 problem), on
 *                        FP32 vectors, with r scaled by a power of two to norm ~1 (so that the
 *                        shrinking residual never leaves the float range) and the result
 *                        scaled back exactly;
 *   x += d,
 * from x = 0 until ||r||_2 <= rtol ||b||_2 (checked on the FP64 residual, so the result meets
 * the same residual criterion as fe_pcg).  maxit bounds the total inner iterations.  The
 * handle's variant is not used.  The FP32 copy of the quadrature data is made on first use.
 * stats: iters = inner iterations, outer_iters = refinement steps, rel_resid = true_rel_resid =
 * final FP64 residual.  Returns FE_ERR_NOT_CONVERGED also when a refinement step fails to reduce
 * the residual. */
int fe_pcg_ir(fe_pa* pa, int op, int pc, const double* dev_b, double* dev_x, double rtol, int maxit,
              double inner_rtol, fe_pcg_stats* stats, void* stream);

/* Batched Jacobi- (or un-) preconditioned CG: nrhs independent systems A_bc x_j = b_j with the
 * same operator (the batched-RHS extension; the paper solves one system), b_j = dev_b + j*ldb,
 * x_j = dev_x + j*ldx (leading dimensions in elements, >= ndofs; 1 <= nrhs <= 1024).  The systems
 * advance in lockstep so that each iteration applies the operator to all search directions in
 * one batched launch (FE_VARIANT_F64, F32X2, F32; the DMMA variant applies them one by one);
 * each keeps its own scalars and stops on its own residual, and the call returns when all have
 * stopped.  Same system, stopping rule and iteration batches (with CUDA-graph replay) as
 * fe_pcg.  stats: NULL or an array of nrhs (iters, residuals per system; seconds and launches of
 * the whole call).  Allocates its work vectors (4 nrhs + 1 of ndofs) per call.  Returns FE_OK
 * when every system converged, else the first failing system's status (see stats). */
int fe_pcg_batched(fe_pa* pa, int op, int pc, int nrhs, const double* dev_b, int64_t ldb,
                   double* dev_x, int64_t ldx, double rtol, int maxit, fe_pcg_stats* stats,
                   void* stream);

/* fe_pcg without any device allocation (the paper has no counterpart: this is a service for
 * callers that cannot allocate).  Some applications give all device memory to their own pool
 * allocator up front, and some latency-critical loops cannot afford the blocking and device
 * synchronisation that cudaMalloc/cudaFree can cause; neither can call a routine that allocates.
 * This entry point solves the same system as fe_pcg, with the same kernels, arguments, stats and
 * status codes, but takes every work vector, reduction partial and flag from one fixed device
 * array compiled into the library: at most 262,144 dofs (FE_PCG_NOALLOC_MAX_DOFS), about 10.5 MB
 * of device memory that every GPU which loads the library keeps until the process exits.  Larger
 * meshes are rejected with FE_ERR_ARG and a message.  It calls no cudaMalloc, cudaFree or other
 * allocating routine (the fe_pa must already exist: fe_pa_setup does allocate).
 *  - The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 *    that device current and caches it; make that first call before any stream capture.
 *    A cudaDeviceReset unloads the library's device image with the context, so the cached
 *    address is stale afterwards: do not call this entry point again in that process after a
 *    reset of that device.
 *  - All calls share the one array, which keeps the last call's contents (the call clears what
 *    must start at zero).  Calls whose GPU work overlaps -- on two streams, or from two host
 *    threads -- race on it and give wrong results: serialise them.
 *  - Like fe_pcg it needs an FP64-accurate variant (FE_ERR_UNSUPPORTED for FE_VARIANT_F32); its
 *    p.Ap comes from a separate FP64 dot-product pass instead of the apply's fused partials (those
 *    would need one more allocated array per handle), and its exit residual uses the FP64
 *    operator.
 * Synchronous, like fe_pcg. */
#define FE_PCG_NOALLOC_MAX_DOFS 262144
int fe_pcg_noalloc(const fe_pa* pa, int op, int pc, const double* dev_b, double* dev_x,
                   double rtol, int maxit, fe_pcg_stats* stats, void* stream);

/* Measurement utility behind the roofline denominators (not part of the operator): runs
 * independent multiply-add chains on every SM of the current device and returns the sustained
 * rate in *tflops (multiply-add = 2 flops; one m8n8k4 DMMA = 512 flops; one m16n8k16 MMA = 4096
 * flops).  Units: FE_PROBE_FP64_FMA, FE_PROBE_FP64_DMMA, FE_PROBE_FP32_FMA, FE_PROBE_F32X2_MAC
 * (the anchored float-float step of the apply, counted as one FP64-equivalent multiply-add),
 * FE_PROBE_BF16_MMA (mma.sync m16n8k16 BF16 with FP32 accumulation, the instruction of the
 * learned preconditioner's kernels), FE_PROBE_FP64_DFMA_DMMA (DFMA chains in half the warps and
 * DMMA chains in the other half at once, both counted: above the DFMA rate only if the two do
 * not share a datapath).  Synchronous; allocates 64 bytes of scratch. */
enum {
  FE_PROBE_FP64_FMA = 0,
  FE_PROBE_FP64_DMMA = 1,
  FE_PROBE_FP32_FMA = 2,
  FE_PROBE_F32X2_MAC = 3,
  FE_PROBE_BF16_MMA = 4,
  FE_PROBE_FP64_DFMA_DMMA = 5
};
int fe_probe_throughput(int unit, double* tflops);

/* ---- Learned element-patch preconditioner and flexible CG (an extension; the paper has no
 * learned component and solves with Jacobi-PCG only).
 *
 * The preconditioner is an additive patch map  z = M(r) = sum_e R_e^T W_e S_e s_e f(x_e / s_e)  with
 *   W_e = diag(1 / number of elements sharing the dof)^(1/2) on element e, 0 on the boundary,
 *   S = diag(A)^(-1/2), x_e = S_e W_e R_e r, s_e = ||x_e||_2, and
 *   f(x) = relu(relu(x W1) W2) W3 + x W0, a bias-free three-layer perceptron D^3 -> width ->
 *   width -> D^3 (D = order + 1) plus a linear skip term, with BF16 weights and activations and
 *   FP32 accumulation on the tensor cores.  With f(x) = S_e^{-1} A_ee^{-1} S_e^{-1} x exactly, M
 *   is the symmetrically weighted additive Schwarz method on element patches.  M is nonlinear
 *   (though positively homogeneous), so it is used inside flexible CG.
 * Training pairs come from the operator itself: for interior elements (in up to 27 classes of
 * elements three apart in each direction, at most 2^28 / D^6 elements), the block A_ee of the
 * assembled matrix on the element's dofs is probed with D^3 applies per class and factored by
 * FP64 Cholesky; f is trained with Adam, to the relative squared error,
 * on pairs x = S_e v, t = S_e^{-1} A_ee^{-1} v scaled by 1/||t||, for v i.i.d. normal, A_ee u for
 * normal u, or W_e r for residuals r of a short Jacobi-FCG run.
 * Built for orders 1..8: the FP64 Cholesky of A_ee runs in one block's shared memory up to
 * order 4 and by 32-column panels in shared memory above; the fused inference kernel covers
 * D^3 <= 128 (orders 1..4), higher orders apply the network by the unfused GEMM path.
 * Handles are library-owned, refer to (do not own) their fe_pa, and are not thread-safe. */
typedef struct fe_lpc fe_lpc;

/* Creates the preconditioner for operator op of pa: He-normal weights W1..W3 (seeded), W0 = 0,
 * the diagonal scalings and the partition-of-unity weights.  width 8..4096, or 0 for the linear
 * patch map f(x) = x W0 (no hidden layers; measured to need fewer FCG iterations than the MLP on
 * these operators, the MLP's nonlinear error acting like preconditioner noise).  Synchronous. */
int fe_lpc_create(fe_pa* pa, int op, int width, uint64_t seed, fe_lpc** out);

/* Number of FP32 master weights: 2 * D^3 * width + width^2 + D^6 (W1 [D^3][width],
 * W2 [width][width], W3 [width][D^3], W0 [D^3][D^3], row-major, packed in that order). */
int fe_lpc_nparams(const fe_lpc* lpc, int64_t* nparams);

/* Runs `steps` Adam steps (beta 0.9 / 0.999, eps 1e-8, learning rate lr) on batches of `batch`
 * pairs drawn from the training set, which is generated on the first call with `reps` pairs per
 * sampled element (0 => 16).  *final_loss (may be NULL) = the relative squared error of the last
 * batch before its step.  Returns FE_ERR_ARG if the mesh has fewer than 3 elements per axis,
 * FE_ERR_BREAKDOWN if a sampled block is not positive
 * definite.  Synchronous. */
int fe_lpc_train(fe_lpc* lpc, int steps, int batch, double lr, int reps, double* final_loss,
                 void* stream);

/* Least-squares fit of the linear term: W = argmin sum ||x W - t||^2 + ridge mean(diag X^T X)
 * ||W||^2 over the whole training set (generated first if needed, `reps` pairs per sampled
 * element, 0 => 16), by the normal equations -- X^T X and X^T T with the BF16 tensor-core GEMM
 * (FP32 accumulation), FP64 Cholesky on the host -- in milliseconds instead of Adam steps; W0 =
 * (W + W^T) / 2, its symmetric part (the scaled local inverse it approximates is symmetric; an
 * antisymmetric remainder from sampling makes flexible CG stall at high coefficient contrast).
 * The other weights are untouched: for width 0 this is the whole preconditioner; for an MLP it
 * is a starting point for fe_lpc_train.  *fit_loss (may be NULL): the relative squared error of
 * W0 on the training set.  Synchronous. */
int fe_lpc_fit_linear(fe_lpc* lpc, double ridge, int reps, double* fit_loss, void* stream);

/* Copies the FP32 master weights (fe_lpc_nparams floats) to host_w (set = 0) or from host_w
 * (set != 0; the BF16 copy is refreshed).  Synchronous. */
int fe_lpc_weights(fe_lpc* lpc, float* host_w, int set);

/* Test hook of the training kernels: for `batch` host rows X (FP32 [batch][D^3], rounded to
 * BF16) and targets T (FP32 [batch][D^3]), runs the forward pass and back-propagation with the
 * current weights and returns the outputs Y (FP32, may be NULL), the gradient of the loss
 * sum ||Y - T||^2 / sum ||T||^2 with respect to the packed weights (FP32, may be NULL) and the
 * loss.  Does not update the weights.  Synchronous. */
int fe_lpc_loss_grad(fe_lpc* lpc, int batch, const float* host_x, const float* host_t,
                     float* host_y, float* host_grad, double* loss);

/* Test hook of the optimiser: for `batch` host rows X (FP32 [batch][D^3], rounded to BF16) and
 * targets T (FP32 [batch][D^3]), runs the forward pass and back-propagation with the current
 * weights and then one Adam step (beta 0.9 / 0.999, eps 1e-8, learning rate lr, the step count
 * advanced by one) -- the kernels of one fe_lpc_train step on a given batch instead of a drawn
 * one.  *loss (may be NULL) = the batch's loss before the step.  Synchronous. */
int fe_lpc_adam_step(fe_lpc* lpc, int batch, const float* host_x, const float* host_t,
                     double lr, double* loss);

/* Test hook of the training-data generator: (re)generates the training set exactly as the first
 * fe_lpc_train call does (probing of A_ee, FP64 Cholesky, residual snapshots, reps pairs per
 * sampled element; reps <= 0 => 16; the BF16/FP32 training copies are replaced) and copies the
 * first min(max_rows, total) pairs to the host in FP64, before their rounding to the training
 * copies: host_elem int32 [rows] the element of each pair, host_x and host_t FP64 [rows][D^3]
 * with t = S_e^-1 A_ee^-1 S_e^-1 x and ||t|| = 1.  *rows gets the count (max_rows = 0: none is
 * copied).  Same errors as fe_lpc_train.  Synchronous. */
int fe_lpc_sample_pairs(fe_lpc* lpc, int reps, int64_t max_rows, int32_t* host_elem,
                        double* host_x, double* host_t, int64_t* rows, void* stream);

/* Checkpoint of a learned preconditioner, so that training resumes where it stopped.  File
 * layout (little-endian): 8 bytes "FELPC001", int32 din (= D^3), int32 width, int64 nparam,
 * int32 Adam step count, int32 0, then nparam FP32 weights (the fe_lpc_weights packing), the
 * nparam FP32 Adam first moments and the nparam FP32 second moments.  fe_lpc_save writes it
 * (FE_ERR_ARG if the file cannot be written); fe_lpc_load reads it into lpc (FE_ERR_ARG on a
 * missing, foreign, truncated file or one of another network shape; the training set is not
 * stored: the next fe_lpc_train regenerates it from the operator, with the same seed the same
 * set).  fe_lpc_checkpoint_info reads only the header, on the host (no device needed); any
 * output may be NULL.  Synchronous. */
int fe_lpc_save(fe_lpc* lpc, const char* path);
int fe_lpc_load(fe_lpc* lpc, const char* path);
int fe_lpc_checkpoint_info(const char* path, int* din, int* width, int64_t* nparam,
                           int* adam_steps);

/* Attaches lpc (built for this pa; NULL detaches) as the preconditioner that fe_pcg uses for
 * pc = FE_PC_LEARNED.  The handle is not owned; fe_lpc_destroy detaches it.  FE_ERR_ARG if lpc
 * was built for another fe_pa. */
int fe_pa_set_learned(fe_pa* pa, fe_lpc* lpc);

/* What fe_fcg continues with once it gives up the network: FE_PC_JACOBI (the default: FCG
 * restarted with Jacobi from the current iterate) or FE_PC_CHEBYSHEV (Chebyshev-PCG on the
 * residual equation).  fe_fcg_ir's inner solves always fall back to Jacobi.  FE_ERR_ARG
 * otherwise. */
int fe_lpc_set_fallback(fe_lpc* lpc, int pc);

/* z = M(r) for FP64 device vectors of length ndofs (z overwritten; z = 0 on the boundary).
 * Asynchronous. */
int fe_lpc_apply(fe_lpc* lpc, const double* dev_r, double* dev_z, void* stream);

/* Inference kernel of the learned preconditioner (fe_lpc_apply, fe_fcg, fe_fcg_ir):
 *   FE_LPC_KERNEL_AUTO      the fastest built kernel as measured on GB300: tcgen05 at width
 *                           256, else the mma.sync fused kernel where it is built, else the
 *                           tcgen05 one, else the unfused GEMM path (the default);
 *   FE_LPC_KERNEL_TCGEN05   fused, 128-element tiles, every layer on the 5th-generation tensor
 *                           cores (tcgen05.mma, FP32 accumulators in tensor memory, weights
 *                           staged by bulk copies; at width 256 the hidden activations stay in
 *                           tensor memory as the next layer's operand); built for width 0, 64
 *                           or 128 with D^3 <= 128 (padded to a multiple of 16), and width 256
 *                           with D^3 <= 64;
 *   FE_LPC_KERNEL_MMA_SYNC  fused, one warp per 16 elements, warp-level mma.sync;
 *   FE_LPC_KERNEL_GEMM      gather kernel, the training path's four BF16 GEMMs, scatter kernel.
 * FE_ERR_UNSUPPORTED if the fused kernel asked for is not built for this order and width.
 * fe_lpc_get_kernel returns the kernel a call uses now (never AUTO) and, when tc_faults is not
 * NULL, whether a tcgen05 launch has given up a bounded wait on the tensor core since the
 * handle was created (synchronous; such a launch leaves z incomplete, and fe_fcg / fe_fcg_ir
 * return FE_ERR_CUDA when it happens during their solve). */
typedef enum {
  FE_LPC_KERNEL_AUTO = 0,
  FE_LPC_KERNEL_TCGEN05 = 1,
  FE_LPC_KERNEL_MMA_SYNC = 2,
  FE_LPC_KERNEL_GEMM = 3
} fe_lpc_kernel;
int fe_lpc_set_kernel(fe_lpc* lpc, int kernel);
int fe_lpc_get_kernel(const fe_lpc* lpc, int* kernel, int* tc_faults);

/* Flexible CG (FCG with one stored direction: beta = -(z.q)/(p.q), alpha = (p.r)/(p.q)) for the
 * same system, arguments and stopping rule as fe_pcg, preconditioned by lpc, or by Jacobi when
 * lpc is NULL.  If the learned preconditioner produces a non-descent direction (z.r <= 0) or the
 * residual stops improving (no 1% gain in 500 iterations, or a 1e4-fold rise) the iteration
 * restarts from the current iterate with Jacobi, or -- after fe_lpc_set_fallback(lpc,
 * FE_PC_CHEBYSHEV) -- hands over to Chebyshev-PCG (fe_pcg_chebyshev with its defaults), which
 * solves A d = (1-m)(b - A x) to the tolerance that meets rtol for x + d, and x += d.  Applies
 * use pa's variant; vectors and inner products are FP64.  stats: outer_iters = 1 + number of
 * such restarts / hand-overs; iters counts both solvers' iterations; with the hand-over also
 * allocates 3 vectors and fe_pcg_chebyshev's workspace.  Synchronous. */
int fe_fcg(fe_pa* pa, int op, fe_lpc* lpc, const double* dev_b, double* dev_x, double rtol,
           int maxit, fe_pcg_stats* stats, void* stream);

/* Mixed-precision iterative refinement with the learned preconditioner (the two extensions
 * combined): outer steps r = (1-m)(b - A x) with the FP64 operator (FE_VARIANT_F64) in FP64
 * vectors; inner flexible CG on FP32 vectors with the FP32 apply (FP32 copy of the quadrature
 * data, made on first use) and lpc applied to FP32 vectors, on r scaled by a power of two to
 * norm ~1, to inner_rtol * ||r|| (0 => 1e-2); x += d (scaled back exactly); until
 * ||r|| <= rtol ||b||, checked on the FP64 residual.  lpc needs an FP32 fused kernel (the
 * mma.sync one at width 0, 64 or 128, or tcgen05; FE_ERR_UNSUPPORTED otherwise).  stats: iters = inner iterations, outer_iters = refinement steps, rel_resid =
 * true_rel_resid = the final FP64-accurate residual.  FE_ERR_NOT_CONVERGED also when a
 * refinement step fails to reduce the residual.  Allocates 2 FP64 and 7 FP32 vectors per call. */
int fe_fcg_ir(fe_pa* pa, int op, fe_lpc* lpc, const double* dev_b, double* dev_x, double rtol,
              int maxit, double inner_rtol, fe_pcg_stats* stats, void* stream);

void fe_lpc_destroy(fe_lpc* lpc);

/* ---- Variable-order spaces (an extension: mixed orders in one mesh) -------------------------
 * One polynomial order per element on the nx x ny x nz structured mesh.  The global space is the
 * continuous piecewise-Q_{p_e} space under the minimum rule, and P of Eq. (1) is the constraint
 * operator that keeps it continuous (Fig. 1's caption: P also carries constraints; the paper
 * gives no construction, so this is a reading):
 *  - entity orders: a cell has its element's order, a face / an edge the smallest order among
 *    the elements containing it; vertices carry one value;
 *  - true dofs: the values at the interior GLL_q nodes of every entity of order q, numbered
 *    vertices first (lexicographic on the (nx+1)(ny+1)(nz+1) lattice), then the x-, y- and
 *    z-directed edges (each family lexicographic on its index box, x fastest; q-1 dofs per edge
 *    by increasing coordinate), then the x-, y- and z-normal faces likewise ((q-1)^2 dofs each,
 *    first in-plane axis fastest: x-normal (y, z), y-normal (x, z), z-normal (x, y)), then the
 *    cells ((p-1)^3 each, x fastest);
 *  - E = G P: an element node takes the value of the function of the entity whose relative
 *    interior holds it (edge: degree-q interpolant of its closure nodes; face: Q_q interpolant of
 *    its closure nodes, whose boundary values come from the bounding edges), evaluated at the
 *    node's GLL_p position.
 * The E-vector holds the elements grouped by ascending order, elements ascending within a group,
 * D^3 nodes per element (a = i + D*(j + D*k)); fe_vspace_layout gives every element's offset.
 * The action is y = E^T blockdiag(A_e) E x: rows of E that are a single weight 1 live in the
 * element map of the fused apply kernel of each order (one persistent launch over all orders,
 * or one launch per order; each order's quadrature data at p+2 Gauss points); the other rows C
 * (nodes constrained by a
 * lower-order neighbour) are applied as [x; C x] before and folded back by C^T after.  Vectors
 * are FP64 of length ntrue. */
typedef struct fe_vspace fe_vspace;

/* host_order: int32 [nx*ny*nz] orders 1..8; host_vertices as for fe_mesh_setup; host_coeff:
 * FP64 [ne] piecewise-constant coefficient or NULL for 1; ops: FE_DIFFUSION | FE_MASS.  Builds
 * the numbering and E on the host, uploads the element map (int32 per E-vector row), C and C^T
 * (CSR: int64 offsets, int32 columns, FP64 weights), two work vectors of ntrue + (rows of C)
 * values, and the per-order partial assembly.  FE_ERR_ARG on a bad order, size or an inverted
 * element; FE_ERR_UNSUPPORTED past 2^31-1 true, local or constrained values.  Synchronous. */
int fe_vspace_setup(int nx, int ny, int nz, const int32_t* host_order,
                    const double* host_vertices, const double* host_coeff, int ops, void* stream,
                    fe_vspace** out);

/* Host-only construction of E (no device, no CUDA call): the numbering, E-vector layout and
 * boundary mask that fe_vspace_setup would build, for inspection and for tests on machines
 * without a GPU.  ntrue, nlocal, nnz: required outputs.  Optional outputs (NULL to skip; call
 * once with NULLs to get the sizes): rowptr int64 [nlocal + 1], cols int32 [nnz] and vals FP64
 * [nnz] (E in CSR, rows in E-vector order; cols and vals together), elem_first int64 [ne],
 * mask uint8 [ntrue].  FE_ERR_ARG on a bad size or order. */
int fe_vspace_host_E(int nx, int ny, int nz, const int32_t* host_order, int64_t* ntrue,
                     int64_t* nlocal, int64_t* nnz, int64_t* rowptr, int32_t* cols, double* vals,
                     int64_t* elem_first, uint8_t* mask);

/* Sizes: true dofs, E-vector length (sum of D_e^3), nonzeros of E; any pointer may be NULL. */
int fe_vspace_sizes(const fe_vspace* vs, int64_t* ntrue, int64_t* nlocal, int64_t* nnz);

/* Size of the constraint part: rows of E that are not a single weight 1 (nodes constrained by a
 * lower-order neighbour), their nonzeros, and the true dofs they touch; any pointer may be NULL. */
int fe_vspace_constraint_sizes(const fe_vspace* vs, int64_t* nrows, int64_t* nnz,
                               int64_t* ntouched);

/* host_first: int64 [ne], the E-vector offset of every element (in element index order). */
int fe_vspace_layout(const fe_vspace* vs, int64_t* host_first);

/* Copies the true-dof boundary mask (uint8 [ntrue], 1 on the cube's boundary) to dev_mask. */
int fe_vspace_boundary_mask(const fe_vspace* vs, uint8_t* dev_mask, void* stream);

/* Selects the arithmetic of every order's apply (as fe_pa_set_variant). */
int fe_vspace_set_variant(fe_vspace* vs, int variant, void* stream);

/* dev_e (FP64 [nlocal]) = E dev_x: the element values of a true-dof vector.  Asynchronous. */
int fe_vspace_prolong(const fe_vspace* vs, const double* dev_x, double* dev_e, void* stream);

/* How fe_vspace_apply runs the element applies: enable != 0 (the default) -- one persistent
 * launch over all orders (thread blocks pull blocks of elements, highest order first, from a
 * device counter), used when every order group has the same FE_VARIANT_F64 or FE_VARIANT_F32X2
 * arithmetic; enable = 0 -- one fused launch per order.  Same results either way. */
int fe_vspace_set_persistent(fe_vspace* vs, int enable);

/* dev_y = E^T blockdiag(A_e) E dev_x for op (no boundary conditions); uses the handle's two
 * work vectors, so calls on one handle must not overlap.  Asynchronous. */
int fe_vspace_apply(const fe_vspace* vs, int op, const double* dev_x, double* dev_y,
                    void* stream);

/* dev_diag (FP64 [ntrue]) = diag(E^T blockdiag(diag A_e) E): every element's own diagonal (the
 * fe_assemble_diagonal of its order) summed with the squared weights of E.  It is the diagonal
 * of E^T A E on every true dof that no element reaches through more than one of its nodes (all
 * but the dofs of the lower-order faces and edges that constrain a higher-order neighbour) and a
 * positive approximation of it on those.  Uses the handle's work vectors.  Asynchronous. */
int fe_vspace_diagonal(const fe_vspace* vs, int op, double* dev_diag, void* stream);

/* Jacobi-PCG on the variable-order space with fe_vspace_diagonal as the Jacobi diagonal: the
 * conventions of fe_pcg (x = 0 start, homogeneous essential conditions on the boundary mask,
 * FP64 vectors, fixed-order reductions, stop at ||r|| <= rtol ||(1-m) b||; stats as fe_pcg's,
 * with the true residual from the handle's variant).  Allocates 5 vectors on the first call (kept
 * with the handle).  FE_ERR_NOT_CONVERGED / FE_ERR_BREAKDOWN / FE_ERR_NAN as fe_pcg.
 * Synchronous. */
int fe_vspace_pcg(fe_vspace* vs, int op, const double* dev_b, double* dev_x, double rtol,
                  int maxit, fe_pcg_stats* stats, void* stream);

/* Batched apply on the variable-order space: dev_y + r ldy = E^T blockdiag(A_e) E (dev_x + r ldx)
 * for r < nrhs (1..1024, ld >= ntrue), all right-hand sides in one persistent launch over all
 * orders (when fe_vspace_set_persistent is on and the arithmetic allows; else one launch per
 * order), each thread block applying every right-hand side to its elements so that the dof map
 * and quadrature data come from L2 after the first.  Uses work vectors of 2 nrhs (ntrue + rows
 * of C) values kept with the handle (allocated on first use, grown when nrhs grows): calls on one
 * handle must not overlap.  Asynchronous. */
int fe_vspace_apply_batched(const fe_vspace* vs, int op, int nrhs, const double* dev_x,
                            int64_t ldx, double* dev_y, int64_t ldy, void* stream);

/* Jacobi-PCG for nrhs systems on the variable-order space in lockstep (the conventions of
 * fe_pcg_batched: each system keeps its own scalars and stops on its own residual; every
 * iteration applies the operator to all search directions with one fe_vspace_apply_batched;
 * iteration batches are replayed as CUDA graphs; deterministic FP64 inner products; true
 * residuals with the FP64 operator; diagonal as fe_vspace_diagonal).  stats: NULL or nrhs
 * entries.  FE_ERR_UNSUPPORTED for the FP32 variant.  Allocates its work vectors per call.
 * Synchronous. */
int fe_vspace_pcg_batched(fe_vspace* vs, int op, int nrhs, const double* dev_b, int64_t ldb,
                          double* dev_x, int64_t ldx, double rtol, int maxit,
                          fe_pcg_stats* stats, void* stream);

/* The learned patch preconditioner on a variable-order space (an extension; the paper has no
 * learned part): one network per order, M(r) = E^T F_X sum_e R_e^T s_e f_p(e)(x_e / s_e) with
 * x_e = R_e F_X E r, s_e = ||x_e||_2, R_e element e's rows of the local vector E r (true dofs
 * and the constrained rows C r), and F_X = (mult_X diag_X)^(-1/2) on the true-dof rows: mult_X
 * the number of element rows of every order that read the row, diag_X the true dof's entry of
 * fe_vspace_diagonal; F_X = 0 on the boundary rows and on every constrained row (the true dofs
 * it interpolates are patch unknowns of the elements that own them); r is taken zero on the
 * boundary.  With one order everywhere M is fe_lpc_apply's operator.
 * fe_vspace_set_learned attaches to the order group `order` a copy of the weights of `trained`
 * (an fe_lpc of that order, trained or fitted on a single-order mesh; the copy is owned by vs
 * and recomputes F_X), or detaches it (trained = NULL); networks of another operator are
 * dropped.  FE_ERR_ARG for an order the space does not contain or a network of another order.
 * Synchronous. */
int fe_vspace_set_learned(fe_vspace* vs, int op, int order, const fe_lpc* trained, void* stream);

/* z = M(r) (FP64 device vectors of length ntrue, z overwritten, 0 on the boundary);
 * FE_ERR_UNSUPPORTED unless every order has a network.  Asynchronous. */
int fe_vspace_lpc_apply(fe_vspace* vs, const double* dev_r, double* dev_z, void* stream);

/* Flexible CG (as fe_fcg) on the variable-order space with M, falling back to Jacobi (the diagonal
 * of fe_vspace_diagonal) when it stalls; FP64 inner products and exit true residual with the
 * FP64 operator.  FE_ERR_UNSUPPORTED unless every order has a network for op, or for the FP32
 * variant.  Same statuses as fe_pcg.  Synchronous. */
int fe_vspace_fcg(fe_vspace* vs, int op, const double* dev_b, double* dev_x, double rtol,
                  int maxit, fe_pcg_stats* stats, void* stream);

void fe_vspace_destroy(fe_vspace* vs);

/* ---- The paper's own operator: the mixed H1 / L2 gradient and divergence blocks ------------
 * Section II-A, Eq. (block-mult) couples an H1 pressure p and an L2 vector velocity u through
 * (grad p, tau) and -(u, grad v); Section III-G applies them in fused partial-assembly kernels.
 * Readings (the paper fixes only the orders, H1 4 and L2 3): H1 of order order_h on the GLL
 * nodes with the structured dof map (the numbering of fe_mesh_setup); L2 of order order_l, one
 * Lagrange basis per element on the order_l + 1 Gauss-Legendre points per axis, three
 * components, layout [e][c][a] with a = i + D_l (j + D_l k), D_l = order_l + 1 (no continuity);
 * Q = order_h + 1 Gauss-Legendre points per axis; the L2 basis used as is on the physical
 * element.  The gradient block is
 *   (G p)_{e,c,a} = sum_q w_q det J (J^-T grad phi_b)_c psi_a p_{g(e,b)},
 * an [ndof_l x ndof_h] operator, and the divergence block is its transpose (the system's
 * -(u, grad v) is -G^T).  The partial assembly stores M_q = w_q det J J^-T (9 FP64 values per
 * element and Gauss point, [e][qz][9][qy][qx]) once; one fused FP64 kernel applies both blocks
 * in one pass over the elements, reading M_q once for both. */
typedef struct fe_mixed fe_mixed;

/* Builds the H1 mesh topology (as fe_mesh_setup with order order_h) and the quadrature data.
 * (order_h, order_l) in {(4, 3) -- the paper's pair --, (2, 1), (3, 3)}, else
 * FE_ERR_UNSUPPORTED; host_vertices as for fe_mesh_setup; FE_ERR_ARG on an inverted element.
 * Synchronous. */
int fe_mixed_setup(int nx, int ny, int nz, int order_h, int order_l, const double* host_vertices,
                   void* stream, fe_mixed** out);

/* H1 dofs ((nx p_h + 1)(ny p_h + 1)(nz p_h + 1)) and L2 values (3 ne D_l^3); either may be NULL. */
int fe_mixed_sizes(const fe_mixed* mx, int64_t* ndof_h, int64_t* ndof_l);

/* dev_gp = G dev_p (FP64 [ndof_l], overwritten) and dev_gtu = G^T dev_u (FP64 [ndof_h], zeroed
 * then scatter-added) in one fused launch; pass dev_p with dev_gp and dev_u with dev_gtu, or
 * NULL for both of a pair to apply one block only.  No aliasing.  Asynchronous. */
int fe_mixed_apply(const fe_mixed* mx, const double* dev_p, const double* dev_u, double* dev_gp,
                   double* dev_gtu, void* stream);

void fe_mixed_destroy(fe_mixed* mx);

void fe_pa_destroy(fe_pa* pa);
void fe_mesh_destroy(fe_mesh* mesh);

/* Message for the calling thread's last non-OK status ("" if none). */
const char* fe_last_error(void);

/* Library version string. */
const char* fe_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FE_H */
