// Launch helpers shared by the per-variant translation units of the fused apply.
#pragma once

#include <algorithm>
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

template <int D, int Q>
inline void fill_tab(const Basis1D& b, TabF32<D, Q>* t) {
  for (int i = 0; i < Q * D; ++i) {
    t->B[i] = (float)b.B[i];
    t->G[i] = (float)b.G[i];
  }
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
  fill_tab<D, Q>(*a.basis, &tab);
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
