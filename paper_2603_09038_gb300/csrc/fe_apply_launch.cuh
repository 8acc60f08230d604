// Launch helpers shared by the per-variant translation units of the fused apply.
#pragma once

#include <mutex>

#include "fe_apply_kernel.cuh"
#include "fe_internal.h"

namespace fe {

// Elements per block: as many as fit in ~96 KB of shared memory (two blocks per SM), a power
// of two, at most 64.
template <int D, int Q, bool DIFF, class T>
constexpr int elems_per_block() {
  constexpr int bytes = ApplyLayout<D, Q, DIFF>::PER_ELEM * (int)sizeof(T);
  int ne = (96 * 1024) / bytes;
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
inline void fill_tab(const Basis1D& b, TabF32x2<D, Q>* t) {
  for (int i = 0; i < Q * D; ++i) {
    const float bh = (float)b.B[i], gh = (float)b.G[i];
    t->Bh[i] = bh;
    t->Bl[i] = (float)(b.B[i] - (double)bh);
    t->Gh[i] = gh;
    t->Gl[i] = (float)(b.G[i] - (double)gh);
  }
}

template <int D, int Q, int NT, bool DIFF, class Ar>
int run_apply(const ApplyArgs& a, cudaStream_t s) {
  using T = typename Ar::T;
  constexpr int NE = elems_per_block<D, Q, DIFF, T>();
  const size_t smem = (size_t)NE * ApplyLayout<D, Q, DIFF>::PER_ELEM * sizeof(T);
  auto kern = k_pa_apply<D, Q, NE, NT, DIFF, Ar>;
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [&] {
    attr_err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (attr_err != cudaSuccess) return cuda_error(attr_err, "cudaFuncSetAttribute(apply)");
  typename Ar::template Tab<D, Q> tab;
  fill_tab<D, Q>(*a.basis, &tab);
  const int64_t nblk = (a.ne + NE - 1) / NE;
  if (nblk == 0) return FE_OK;
  kern<<<(unsigned int)nblk, NT, smem, s>>>(a.map, a.qd, a.x, a.y, a.ne, a.skip, tab);
  return cuda_error(cudaGetLastError(), "apply kernel launch");
}

// Dispatch on the order for the default rule Q = p + 2.
template <int NT, class Ar>
int dispatch_order(int op, const ApplyArgs& a, cudaStream_t s) {
  const bool diff = (op == FE_DIFFUSION);
  if (a.Q != a.p + 2) return set_error(FE_ERR_UNSUPPORTED, "only q1d = order + 2 is built");
#define FE_CASE(P)                                                                  \
  case P:                                                                           \
    return diff ? run_apply<P + 1, P + 2, NT, true, Ar>(a, s)                       \
                : run_apply<P + 1, P + 2, NT, false, Ar>(a, s);
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
