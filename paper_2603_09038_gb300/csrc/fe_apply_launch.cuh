// Launch helpers shared by the per-variant translation units of the fused apply.
#pragma once

#include <algorithm>
#include <cstring>
#include <cmath>
#include <mutex>

#include "fe_apply_kernel.cuh"
#include "fe_internal.h"

namespace fe {

// Launch shape per arithmetic variant: threads per block, shared-memory budget per block (the
// elements per block follow from it) and the smallest D from which the z phase re-reads its
// inputs from shared memory instead of holding them in registers.  The defaults come from
// sweeps on GB300; the macros exist for tuning builds.
#ifndef FE_F64_NT
#define FE_F64_NT 128
#endif
#ifndef FE_F64_SMEM
#define FE_F64_SMEM (96 * 1024)
#endif
#ifndef FE_F64_REREAD_D
#define FE_F64_REREAD_D 5
#endif
#ifndef FE_F64_MINB
#define FE_F64_MINB 1
#endif
#ifndef FE_F32X2_MINB
#define FE_F32X2_MINB 2
#endif
#ifndef FE_F32X2_NT
#define FE_F32X2_NT 256
#endif
#ifndef FE_F32X2_SMEM
#define FE_F32X2_SMEM (96 * 1024)
#endif
#ifndef FE_F32X2_REREAD_D
#define FE_F32X2_REREAD_D 2
#endif

// Launch shapes (threads per block, shared-memory budget -> elements per block, minimum blocks
// per SM for the register allocation).  Each arithmetic has a few built shapes; shape 0 is the
// default and fe_pa_autotune times the others.
template <int NT_, int SMEM_, int MINB_>
struct Shape {
  static constexpr int NT = NT_, SMEM = SMEM_, MINB = MINB_;
};
template <class Ar, int I>
struct ApplyShape;
template <class Ar>
struct ApplyShapeCount {
  static constexpr int N = 1;
};

template <class Ar>
struct ApplyTuning;
// SPLIT: a separate single-right-hand-side instantiation (the batch loop cost the
// memory-latency-bound FP32 kernel ~20 %; the ALU-bound variants do not notice it).
template <>
struct ApplyTuning<ArF64> {
  static constexpr int NT = FE_F64_NT, SMEM = FE_F64_SMEM, REREAD_D = FE_F64_REREAD_D,
                       MINB = FE_F64_MINB;
  static constexpr bool SPLIT = false;
};
#ifndef FE_F32_NT
#define FE_F32_NT 256
#endif
#ifndef FE_F32_SMEM
#define FE_F32_SMEM (48 * 1024)
#endif
#ifndef FE_F32_MINB
#define FE_F32_MINB 2
#endif
template <>
struct ApplyTuning<ArF32> {
  static constexpr int NT = FE_F32_NT, SMEM = FE_F32_SMEM, REREAD_D = 2, MINB = FE_F32_MINB;
  static constexpr bool SPLIT = true;
};
template <bool A, bool L>
struct ApplyTuning<ArF32x2T<A, L>> {
  static constexpr int NT = FE_F32X2_NT, SMEM = FE_F32X2_SMEM, REREAD_D = FE_F32X2_REREAD_D,
                       MINB = FE_F32X2_MINB;
  static constexpr bool SPLIT = false;
};

template <>
struct ApplyShape<ArF64, 0> : Shape<FE_F64_NT, FE_F64_SMEM, FE_F64_MINB> {};
template <>
struct ApplyShape<ArF64, 1> : Shape<128, 48 * 1024, 3> {};
template <>
struct ApplyShape<ArF64, 2> : Shape<256, 96 * 1024, 1> {};
template <>
struct ApplyShapeCount<ArF64> {
  static constexpr int N = 3;
};
template <bool A, bool L>
struct ApplyShape<ArF32x2T<A, L>, 0> : Shape<FE_F32X2_NT, FE_F32X2_SMEM, FE_F32X2_MINB> {};
template <bool A, bool L>
struct ApplyShape<ArF32x2T<A, L>, 1> : Shape<128, 48 * 1024, 4> {};
template <bool A, bool L>
struct ApplyShape<ArF32x2T<A, L>, 2> : Shape<256, 48 * 1024, 2> {};
template <bool A, bool L>
struct ApplyShapeCount<ArF32x2T<A, L>> {
  static constexpr int N = 3;
};
template <>
struct ApplyShape<ArF32, 0> : Shape<FE_F32_NT, FE_F32_SMEM, FE_F32_MINB> {};
static_assert(ApplyShapeCount<ArF64>::N == kShapesF64 &&
                  ApplyShapeCount<ArF32x2T<true, true>>::N == kShapesF32x2,
              "shape counts of fe_internal.h out of date");

// Elements per block: as many as fit in the shape's shared-memory budget, a power of two,
// at most 64.
template <int D, int Q, bool DIFF, class T, int SMEM, bool RR>
constexpr int elems_per_block() {
  constexpr int bytes = ApplyLayout<D, Q, DIFF, (int)sizeof(T), RR>::PER_ELEM * (int)sizeof(T);
  int ne = SMEM / bytes;
  int p2 = 1;
  while (p2 * 2 <= ne && p2 < 64) p2 *= 2;
  return p2;
}

template <int D, int Q>
inline void fill_tab(const Basis1D& b, TabF64<D, Q>* t) {
  for (int i = 0; i < Q * D; ++i) {
    t->B[i] = b.B[i];
    t->G[i] = b.G[i];
  }
}

// The tables and their even-odd halves (eo::fill).
template <class R, int D, int Q>
inline void fill_tab(const Basis1D& b, TabEO<R, D, Q>* t) {
  eo::fill(b.B, b.G, t);
}

template <int D, int Q>
inline void fill_tab(const Basis1D& b, TabF32x2<D, Q>* t) {
  for (int i = 0; i < Q * D; ++i) {
    const float bh = (float)b.B[i], gh = (float)b.G[i];
    t->Bh[i] = bh;
    t->Bl[i] = (float)(b.B[i] - (double)bh);
    t->Gh[i] = gh;
    t->Gl[i] = (float)(b.G[i] - (double)gh);
  }
  // largest absolute row (forward use) and column (transposed use) sums of the high words,
  // rounded up, for the anchors of the float-float dot products
  double rB = 0, rG = 0, cB = 0, cG = 0;
  for (int q = 0; q < Q; ++q) {
    double sb = 0, sg = 0;
    for (int d = 0; d < D; ++d) {
      sb += std::fabs((double)t->Bh[q * D + d]);
      sg += std::fabs((double)t->Gh[q * D + d]);
    }
    rB = std::max(rB, sb);
    rG = std::max(rG, sg);
  }
  for (int d = 0; d < D; ++d) {
    double sb = 0, sg = 0;
    for (int q = 0; q < Q; ++q) {
      sb += std::fabs((double)t->Bh[q * D + d]);
      sg += std::fabs((double)t->Gh[q * D + d]);
    }
    cB = std::max(cB, sb);
    cG = std::max(cG, sg);
  }
  const double up = 1.0 + 1e-6;
  t->rB = (float)(rB * up);
  t->rG = (float)(rG * up);
  t->cB = (float)(cB * up);
  t->cG = (float)(cG * up);
}

template <int D, int Q, bool DIFF, class Ar, class VT, bool MULTI, class SH>
int launch_kernel(const ApplyArgs& a, cudaStream_t s) {
  using T = typename Ar::T;
  using Tune = ApplyTuning<Ar>;
  constexpr int NT = SH::NT;
  constexpr bool RR = (D >= Tune::REREAD_D);
  constexpr int NE = elems_per_block<D, Q, DIFF, T, SH::SMEM, RR>();
  if (a.elems_per_block) *a.elems_per_block = NE;
  if (a.threads_per_block) *a.threads_per_block = NT;
  const size_t smem = (size_t)NE * ApplyLayout<D, Q, DIFF, (int)sizeof(T), RR>::PER_ELEM * sizeof(T);
  auto kern = k_pa_apply<D, Q, NE, NT, DIFF, Ar, (D >= Tune::REREAD_D), SH::MINB, VT, MULTI>;
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [&] {
    attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (attr_err != cudaSuccess) return cuda_error(attr_err, "cudaFuncSetAttribute(apply)");
  typename Ar::template Tab<D, Q> tab;
  fill_tab(*a.basis, &tab);
  const int64_t nblk = (a.ne + NE - 1) / NE;
  if (a.blocks) *a.blocks = nblk;
  if (nblk == 0 || a.query_only) return FE_OK;
  if (Ar::kScaled && a.qscale == nullptr)
    return set_error(FE_ERR_ARG, "apply: float-pair quadrature data without its scales");
  kern<<<(unsigned int)nblk, NT, smem, s>>>(a.map, reinterpret_cast<const typename Ar::QdT*>(a.qd),
                                            a.qscale, a.qshift, reinterpret_cast<const VT*>(a.x),
                                            reinterpret_cast<VT*>(a.y), a.ne, a.skip, a.dot_part,
                                            a.nrhs, a.ldx, a.ldy, tab);
  return cuda_error(cudaGetLastError(), "apply kernel launch");
}

template <int D, int Q, bool DIFF, class Ar, class VT, class SH>
int run_shape(const ApplyArgs& a, cudaStream_t s) {
  if constexpr (ApplyTuning<Ar>::SPLIT) {
    if (a.nrhs == 1) return launch_kernel<D, Q, DIFF, Ar, VT, false, SH>(a, s);
  }
  return launch_kernel<D, Q, DIFF, Ar, VT, true, SH>(a, s);
}

template <int D, int Q, bool DIFF, class Ar, class VT = double>
int run_apply(const ApplyArgs& a, cudaStream_t s) {
  constexpr int N = ApplyShapeCount<Ar>::N;
  if (a.shape < 0 || a.shape >= N) return set_error(FE_ERR_ARG, "apply: no such launch shape");
  if constexpr (N > 2)
    if (a.shape == 2) return run_shape<D, Q, DIFF, Ar, VT, ApplyShape<Ar, (N > 2 ? 2 : 0)>>(a, s);
  if constexpr (N > 1)
    if (a.shape == 1) return run_shape<D, Q, DIFF, Ar, VT, ApplyShape<Ar, (N > 1 ? 1 : 0)>>(a, s);
  return run_shape<D, Q, DIFF, Ar, VT, ApplyShape<Ar, 0>>(a, s);
}

// Dispatch on the order for the default rule Q = p + 2 (Ar may depend on the order through
// ArForOrder).
template <class Ar, int P>
struct ArForOrder {
  using type = Ar;
};

// Float-float accumulation scheme per order, from the measured worst-case error against the FP64
// apply (whole ~25 M dof meshes, random x): anchored sums with lazy normalisation up to p = 3
// (~1.3e-13), anchored with normalisation for p = 4, 5 (<= 2.1e-13), compensated sums for
// p >= 6, where the anchored error reached 4.6e-13 (p = 6) to 5.7e-13 (p = 7) -- the
// compensated sums stay near 3e-14, well inside the 1e-12 parity bar.
template <int P>
struct ArForOrder<ArF32x2, P> {
  using type = ArF32x2T<(P <= 5), (P <= 3)>;
};

// One order's apply, both operators, FP64 vectors.  The float-float orders are instantiated in
// several translation units (fe_apply_f32x2_p*.cu) so that they compile in parallel.
template <class Ar, int P>
int apply_order(int op, const ApplyArgs& a, cudaStream_t s) {
  using A = typename ArForOrder<Ar, P>::type;
  return op == FE_DIFFUSION ? run_apply<P + 1, P + 2, true, A, double>(a, s)
                            : run_apply<P + 1, P + 2, false, A, double>(a, s);
}

template <class Ar, class VT = double>
int dispatch_order(int op, const ApplyArgs& a, cudaStream_t s) {
  const bool diff = (op == FE_DIFFUSION);
  if (a.Q != a.p + 2) return set_error(FE_ERR_UNSUPPORTED, "only q1d = order + 2 is built");
#define FE_CASE(P)                                                                  \
  case P:                                                                           \
    return diff ? run_apply<P + 1, P + 2, true, typename ArForOrder<Ar, P>::type, VT>(a, s) \
                : run_apply<P + 1, P + 2, false, typename ArForOrder<Ar, P>::type, VT>(a, s);
  switch (a.p) {
    FE_CASE(1)
    FE_CASE(2)
    FE_CASE(3)
    FE_CASE(4)
    FE_CASE(5)
    FE_CASE(6)
    FE_CASE(7)
    FE_CASE(8)
    default:
      return set_error(FE_ERR_UNSUPPORTED, "order out of range 1..8");
  }
#undef FE_CASE
}

}  // namespace fe

namespace fe {

// ---- Persistent multi-order apply (a variable-order space): one launch applies every order
// group.  Work items are blocks of elements of one order (the per-order kernel's element blocks);
// the items of the highest order come first and each thread block pulls the next item from a
// device counter until none is left, so the order groups share one grid and its tail.

// 1D tables of every order (entries of absent orders are unused).
template <class Base>
struct MultiTabs {
  typename ArForOrder<Base, 1>::type::template Tab<2, 3> t1;
  typename ArForOrder<Base, 2>::type::template Tab<3, 4> t2;
  typename ArForOrder<Base, 3>::type::template Tab<4, 5> t3;
  typename ArForOrder<Base, 4>::type::template Tab<5, 6> t4;
  typename ArForOrder<Base, 5>::type::template Tab<6, 7> t5;
  typename ArForOrder<Base, 6>::type::template Tab<7, 8> t6;
  typename ArForOrder<Base, 7>::type::template Tab<8, 9> t7;
  typename ArForOrder<Base, 8>::type::template Tab<9, 10> t8;
};

template <class Base, bool DIFF, int SMEM, int P>
struct MultiOrder {
  using Ar = typename ArForOrder<Base, P>::type;
  static constexpr bool RR = (P + 1 >= ApplyTuning<Ar>::REREAD_D);
  static constexpr int NE = elems_per_block<P + 1, P + 2, DIFF, typename Ar::T, SMEM, RR>();
  static constexpr size_t BYTES = (size_t)NE *
      ApplyLayout<P + 1, P + 2, DIFF, (int)sizeof(typename Ar::T), RR>::PER_ELEM *
      sizeof(typename Ar::T);
};

template <class Base, bool DIFF, int SMEM>
constexpr size_t multi_smem() {
  size_t m = 0;
  const size_t b[8] = {MultiOrder<Base, DIFF, SMEM, 1>::BYTES, MultiOrder<Base, DIFF, SMEM, 2>::BYTES,
                       MultiOrder<Base, DIFF, SMEM, 3>::BYTES, MultiOrder<Base, DIFF, SMEM, 4>::BYTES,
                       MultiOrder<Base, DIFF, SMEM, 5>::BYTES, MultiOrder<Base, DIFF, SMEM, 6>::BYTES,
                       MultiOrder<Base, DIFF, SMEM, 7>::BYTES, MultiOrder<Base, DIFF, SMEM, 8>::BYTES};
  for (int i = 0; i < 8; ++i) m = b[i] > m ? b[i] : m;
  return m;
}

template <class Base, bool DIFF, int SMEM>
int multi_elems(int p) {
  switch (p) {
    case 1: return MultiOrder<Base, DIFF, SMEM, 1>::NE;
    case 2: return MultiOrder<Base, DIFF, SMEM, 2>::NE;
    case 3: return MultiOrder<Base, DIFF, SMEM, 3>::NE;
    case 4: return MultiOrder<Base, DIFF, SMEM, 4>::NE;
    case 5: return MultiOrder<Base, DIFF, SMEM, 5>::NE;
    case 6: return MultiOrder<Base, DIFF, SMEM, 6>::NE;
    case 7: return MultiOrder<Base, DIFF, SMEM, 7>::NE;
    case 8: return MultiOrder<Base, DIFF, SMEM, 8>::NE;
    default: return 0;
  }
}

template <class Base, bool DIFF, int NT, int SMEM, int P>
__device__ __forceinline__ void multi_body(const MultiGroups& g, int gi, int64_t blk,
                                           const double* __restrict__ x, double* __restrict__ y,
                                           int nrhs, int64_t ldx, int64_t ldy,
                                           const typename MultiOrder<Base, DIFF, SMEM, P>::Ar::template Tab<P + 1, P + 2>& tab,
                                           unsigned char* smem, int* wexp) {
  using MO = MultiOrder<Base, DIFF, SMEM, P>;
  using Ar = typename MO::Ar;
  pa_apply_block<P + 1, P + 2, MO::NE, NT, DIFF, Ar, MO::RR, double, true>(
      g.map[gi], reinterpret_cast<const typename Ar::QdT*>(g.qd[gi]), g.qscale[gi], 0, x, y,
      g.ne[gi], blk, false, nrhs, ldx, ldy, tab, smem, wexp);
}

template <class Base, bool DIFF, int NT, int MINB, int SMEM>
__global__ void __launch_bounds__(NT, MINB) k_pa_apply_multi(const MultiGroups g,
                                                            const double* __restrict__ x,
                                                            double* __restrict__ y,
                                                            int* __restrict__ counter, int nrhs,
                                                            int64_t ldx, int64_t ldy,
                                                            const MultiTabs<Base> tabs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int wexp[NT / 32];
  __shared__ int s_item;
  const int total = (int)g.first_item[g.n];
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();  // every thread has read the item before thread 0 fetches the next one
    if (item >= total) break;
    int gi = 0;
    while (gi + 1 < g.n && item >= g.first_item[gi + 1]) ++gi;
    const int64_t blk = item - g.first_item[gi];
    switch (g.order[gi]) {
      case 1: multi_body<Base, DIFF, NT, SMEM, 1>(g, gi, blk, x, y, nrhs, ldx, ldy, tabs.t1, smem_raw, wexp); break;
      case 2: multi_body<Base, DIFF, NT, SMEM, 2>(g, gi, blk, x, y, nrhs, ldx, ldy, tabs.t2, smem_raw, wexp); break;
      case 3: multi_body<Base, DIFF, NT, SMEM, 3>(g, gi, blk, x, y, nrhs, ldx, ldy, tabs.t3, smem_raw, wexp); break;
      case 4: multi_body<Base, DIFF, NT, SMEM, 4>(g, gi, blk, x, y, nrhs, ldx, ldy, tabs.t4, smem_raw, wexp); break;
      case 5: multi_body<Base, DIFF, NT, SMEM, 5>(g, gi, blk, x, y, nrhs, ldx, ldy, tabs.t5, smem_raw, wexp); break;
      case 6: multi_body<Base, DIFF, NT, SMEM, 6>(g, gi, blk, x, y, nrhs, ldx, ldy, tabs.t6, smem_raw, wexp); break;
      case 7: multi_body<Base, DIFF, NT, SMEM, 7>(g, gi, blk, x, y, nrhs, ldx, ldy, tabs.t7, smem_raw, wexp); break;
      default: multi_body<Base, DIFF, NT, SMEM, 8>(g, gi, blk, x, y, nrhs, ldx, ldy, tabs.t8, smem_raw, wexp); break;
    }
  }
}

template <class Base>
void fill_multi_tabs(const Basis1D* const* basis, MultiTabs<Base>* t) {
  std::memset(t, 0, sizeof(*t));
  if (basis[0]) fill_tab(*basis[0], &t->t1);
  if (basis[1]) fill_tab(*basis[1], &t->t2);
  if (basis[2]) fill_tab(*basis[2], &t->t3);
  if (basis[3]) fill_tab(*basis[3], &t->t4);
  if (basis[4]) fill_tab(*basis[4], &t->t5);
  if (basis[5]) fill_tab(*basis[5], &t->t6);
  if (basis[6]) fill_tab(*basis[6], &t->t7);
  if (basis[7]) fill_tab(*basis[7], &t->t8);
}

// One persistent launch over the groups of g for nrhs right-hand sides x + r ldx -> y + r ldy (y
// zeroed by the caller; counter: one device int, zeroed here).  basis[p - 1]: the 1D tables of
// order p (NULL where absent).
template <class Base, bool DIFF>
int launch_multi(const MultiGroups& g, const Basis1D* const* basis, const double* x, double* y,
                 int* counter, int nrhs, int64_t ldx, int64_t ldy, cudaStream_t s) {
  using SH = ApplyShape<typename ArForOrder<Base, 1>::type, 0>;
  constexpr size_t smem = multi_smem<Base, DIFF, SH::SMEM>();
  auto kern = k_pa_apply_multi<Base, DIFF, SH::NT, SH::MINB, SH::SMEM>;
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  static int grid_cap = 0;
  std::call_once(once, [&] {
    attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 0, dev = 0, sms = 0;
    if (attr_err == cudaSuccess)
      attr_err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, SH::NT, smem);
    if (attr_err == cudaSuccess) attr_err = cudaGetDevice(&dev);
    if (attr_err == cudaSuccess)
      attr_err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    grid_cap = (occ > 0 ? occ : 1) * (sms > 0 ? sms : 1);
  });
  if (attr_err != cudaSuccess) return cuda_error(attr_err, "multi-order apply: setup");
  const int64_t total = g.first_item[g.n];
  if (total == 0) return FE_OK;
  MultiTabs<Base> tabs;
  fill_multi_tabs<Base>(basis, &tabs);
  cudaError_t err = cudaMemsetAsync(counter, 0, sizeof(int), s);
  if (err != cudaSuccess) return cuda_error(err, "multi-order apply: counter");
  const int grid = (int)(total < grid_cap ? total : grid_cap);
  kern<<<grid, SH::NT, smem, s>>>(g, x, y, counter, nrhs, ldx, ldy, tabs);
  return cuda_error(cudaGetLastError(), "multi-order apply launch");
}

}  // namespace fe
