// Variable-order spaces: one polynomial order per element, kept continuous by the minimum rule.
//
// Eq. (1) reads A = P^T G^T B^T D B G P; with one order P is the identity on one GPU, with
// several it is the constraint operator (Fig. 1's caption).  The space and its numbering are
// documented with fe_vspace_setup in fe.h.  Here E = G P is built on the host once, row by row,
// by evaluating the entity functions at every element node.  Most rows are a single weight 1 (a
// node that is itself a true dof); they become entries of an ordinary element map.  The other
// rows ("constrained": nodes on faces and edges shared with a lower order) form a sparse matrix
// C, and the map sends their nodes to ntrue + c.  An apply is then
//   X = [x; C x] (a copy and a CSR pass over the constrained rows only),
//   Y = sum_g A_g X for every order g present (the fused PA kernel of that order, gathering X and
//       scatter-adding into Y through the group's map; Y zeroed once),
//   y = Y[0, ntrue) + C^T Y[ntrue, ...) (a copy and the transpose over the true dofs C touches,
//       one thread per such dof, fixed order).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <exception>
#include <new>
#include <thread>
#include <vector>

#include "fe_f2.h"
#include "fe_internal.h"

using namespace fe;

namespace {
#include "fe_solver_common.cuh"
}  // namespace

namespace {

constexpr int kRowCap = (kMaxD) * (kMaxD);  // distinct columns of one E row: a face closure

struct Row {
  int n = 0;
  int64_t col[kRowCap];
  double w[kRowCap];
  void add(int64_t c, double v) {
    if (v == 0.0) return;
    for (int t = 0; t < n; ++t)
      if (col[t] == c) {
        w[t] += v;
        return;
      }
    col[n] = c;
    w[n] = v;
    ++n;
  }
};

// l_m(x) of the Lagrange basis on nodes t[0..n-1] (product formula).  A point within 1e-13 of a
// node is that node (l_m = delta): GLL nodes of different orders coincide at 0, 1/2 and 1, and
// their separately computed values may differ in the last bit.
void lagrange_at(const double* t, int n, double x, double* L) {
  for (int k = 0; k < n; ++k)
    if (std::fabs(x - t[k]) <= 1e-13) {
      for (int m = 0; m < n; ++m) L[m] = m == k ? 1.0 : 0.0;
      return;
    }
  for (int m = 0; m < n; ++m) {
    double v = 1.0;
    for (int k = 0; k < n; ++k)
      if (k != m) v *= (x - t[k]) / (t[m] - t[k]);
    L[m] = v;
  }
}

struct Topo {
  int n[3] = {0, 0, 0};
  int64_t ne = 0, nv = 0, ntrue = 0;
  std::vector<int> ord;                 // [ne]
  int64_t ebox[3][3], fbox[3][3];       // index boxes (x, y, z extents) of edges / faces per axis
  std::vector<uint8_t> eq[3], fq[3];    // entity orders
  std::vector<int64_t> efirst[3], ffirst[3], cfirst;
  double gll[kMaxOrder + 1][kMaxD];     // GLL nodes on [0, 1] of every order

  int64_t lin(const int64_t* box, const int64_t* i) const {
    return i[0] + box[0] * (i[1] + box[1] * i[2]);
  }
  int64_t vertex(const int64_t* i) const {
    return i[0] + (int64_t)(n[0] + 1) * (i[1] + (int64_t)(n[1] + 1) * i[2]);
  }
  int cell_order(int64_t x, int64_t y, int64_t z) const {
    if (x < 0 || y < 0 || z < 0 || x >= n[0] || y >= n[1] || z >= n[2]) return 1 << 20;
    return ord[x + (int64_t)n[0] * (y + (int64_t)n[1] * z)];
  }

  // Value of the d-directed edge at index idx, at coordinate x in [0, 1] along it, times w.
  void add_edge(int d, const int64_t* idx, double x, double w, Row& r) const {
    const int q = eq[d][lin(ebox[d], idx)];
    double L[kMaxD];
    lagrange_at(gll[q], q + 1, x, L);
    for (int m = 0; m <= q; ++m) {
      const double lw = w * L[m];
      if (lw == 0.0) continue;
      if (m == 0) {
        r.add(vertex(idx), lw);
      } else if (m == q) {
        int64_t hi[3] = {idx[0], idx[1], idx[2]};
        ++hi[d];
        r.add(vertex(hi), lw);
      } else {
        r.add(efirst[d][lin(ebox[d], idx)] + m - 1, lw);
      }
    }
  }

  // Value of the d-normal face at index idx, at in-plane coordinates (xs, xt), times w.
  void add_face(int d, const int64_t* idx, double xs, double xt, double w, Row& r) const {
    const int u = d == 0 ? 1 : 0, v = d == 2 ? 1 : 2;
    const int64_t f = lin(fbox[d], idx);
    const int q = fq[d][f];
    double Lu[kMaxD], Lv[kMaxD];
    lagrange_at(gll[q], q + 1, xs, Lu);
    lagrange_at(gll[q], q + 1, xt, Lv);
    for (int b = 0; b <= q; ++b) {
      for (int a = 0; a <= q; ++a) {
        const double lw = w * Lu[a] * Lv[b];
        if (lw == 0.0) continue;
        const bool ia = a > 0 && a < q, ib = b > 0 && b < q;
        if (ia && ib) {
          r.add(ffirst[d][f] + (a - 1) + (int64_t)(q - 1) * (b - 1), lw);
        } else if (!ia) {  // on the v-directed edge at u = a / q (corners included)
          int64_t e[3] = {idx[0], idx[1], idx[2]};
          e[u] += (a == q);
          add_edge(v, e, gll[q][b], lw, r);
        } else {           // on the u-directed edge at v = b / q
          int64_t e[3] = {idx[0], idx[1], idx[2]};
          e[v] += (b == q);
          add_edge(u, e, gll[q][a], lw, r);
        }
      }
    }
  }

  // Row of E for node (i, j, k) of element e.
  void node_row(int64_t e, int i, int j, int k, Row& r) const {
    r.n = 0;
    const int p = ord[e];
    const int64_t c[3] = {e % n[0], (e / n[0]) % n[1], e / ((int64_t)n[0] * n[1])};
    const int ijk[3] = {i, j, k};
    bool fixed[3];
    int64_t pos[3];
    int nb = 0;
    for (int a = 0; a < 3; ++a) {
      fixed[a] = ijk[a] == 0 || ijk[a] == p;
      pos[a] = c[a] + (ijk[a] == p);
      nb += fixed[a];
    }
    if (nb == 3) {
      r.add(vertex(pos), 1.0);
    } else if (nb == 0) {
      r.add(cfirst[e] + (i - 1) + (int64_t)(p - 1) * ((j - 1) + (int64_t)(p - 1) * (k - 1)), 1.0);
    } else if (nb == 2) {
      const int d = !fixed[0] ? 0 : (!fixed[1] ? 1 : 2);
      int64_t idx[3] = {pos[0], pos[1], pos[2]};
      idx[d] = c[d];
      add_edge(d, idx, gll[p][ijk[d]], 1.0, r);
    } else {
      const int d = fixed[0] ? 0 : (fixed[1] ? 1 : 2);
      const int u = d == 0 ? 1 : 0, v = d == 2 ? 1 : 2;
      int64_t idx[3] = {c[0], c[1], c[2]};
      idx[d] = pos[d];
      add_face(d, idx, gll[p][ijk[u]], gll[p][ijk[v]], 1.0, r);
    }
    // contributions that cancel leave round-off (~1e-17) where the exact weight is 0: drop them
    int kept = 0;
    for (int t = 0; t < r.n; ++t)
      if (std::fabs(r.w[t]) > 1e-13) {
        r.col[kept] = r.col[t];
        r.w[kept] = r.w[t];
        ++kept;
      }
    r.n = kept;
  }

  bool on_boundary_edge(int d, const int64_t* idx) const {
    for (int a = 0; a < 3; ++a)
      if (a != d && (idx[a] == 0 || idx[a] == n[a])) return true;
    return false;
  }
};

// Entity orders and the numbering; false if an order is out of range.
bool build_topology(int nx, int ny, int nz, const int32_t* order, Topo& T) {
  T.n[0] = nx;
  T.n[1] = ny;
  T.n[2] = nz;
  T.ne = (int64_t)nx * ny * nz;
  T.ord.assign(order, order + T.ne);
  for (int p : T.ord)
    if (p < 1 || p > kMaxOrder) return false;
  for (int q = 1; q <= kMaxOrder; ++q) {
    Basis1D b;
    if (!make_basis_1d(q, q + 2, &b)) return false;
    for (int m = 0; m <= q; ++m) T.gll[q][m] = b.nodes[m];
  }
  T.nv = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  int64_t off = T.nv;
  for (int d = 0; d < 3; ++d) {
    for (int a = 0; a < 3; ++a) T.ebox[d][a] = T.n[a] + (a == d ? 0 : 1);
    const int64_t cnt = T.ebox[d][0] * T.ebox[d][1] * T.ebox[d][2];
    T.eq[d].resize(cnt);
    T.efirst[d].resize(cnt);
    int64_t i[3];
    for (i[2] = 0; i[2] < T.ebox[d][2]; ++i[2])
      for (i[1] = 0; i[1] < T.ebox[d][1]; ++i[1])
        for (i[0] = 0; i[0] < T.ebox[d][0]; ++i[0]) {
          int q = 1 << 20;
          for (int s = 0; s < 2; ++s)
            for (int t = 0; t < 2; ++t) {
              int64_t c[3] = {i[0], i[1], i[2]};
              int k = 0;
              for (int a = 0; a < 3; ++a)
                if (a != d) c[a] -= (k++ == 0 ? s : t);
              q = std::min(q, T.cell_order(c[0], c[1], c[2]));
            }
          const int64_t l = T.lin(T.ebox[d], i);
          T.eq[d][l] = (uint8_t)q;
          T.efirst[d][l] = off;
          off += q - 1;
        }
  }
  for (int d = 0; d < 3; ++d) {
    for (int a = 0; a < 3; ++a) T.fbox[d][a] = T.n[a] + (a == d ? 1 : 0);
    const int64_t cnt = T.fbox[d][0] * T.fbox[d][1] * T.fbox[d][2];
    T.fq[d].resize(cnt);
    T.ffirst[d].resize(cnt);
    int64_t i[3];
    for (i[2] = 0; i[2] < T.fbox[d][2]; ++i[2])
      for (i[1] = 0; i[1] < T.fbox[d][1]; ++i[1])
        for (i[0] = 0; i[0] < T.fbox[d][0]; ++i[0]) {
          int64_t c[3] = {i[0], i[1], i[2]};
          const int q0 = T.cell_order(c[0], c[1], c[2]);
          --c[d];
          const int q = std::min(q0, T.cell_order(c[0], c[1], c[2]));
          const int64_t l = T.lin(T.fbox[d], i);
          T.fq[d][l] = (uint8_t)q;
          T.ffirst[d][l] = off;
          off += (int64_t)(q - 1) * (q - 1);
        }
  }
  T.cfirst.resize(T.ne);
  for (int64_t e = 0; e < T.ne; ++e) {
    T.cfirst[e] = off;
    off += (int64_t)(T.ord[e] - 1) * (T.ord[e] - 1) * (T.ord[e] - 1);
  }
  T.ntrue = off;
  return true;
}

// Runs f(begin, end) over [0, n) on the host's cores.
template <class F>
void parallel_for(int64_t n, F f) {
  const int nt = (int)std::max(1u, std::min(std::thread::hardware_concurrency(), 32u));
  if (n < 4096 || nt == 1) {
    f((int64_t)0, n);
    return;
  }
  std::vector<std::thread> th;
  const int64_t chunk = (n + nt - 1) / nt;
  for (int t = 0; t < nt; ++t) {
    const int64_t b = t * chunk, e = std::min(n, b + chunk);
    if (b < e) th.emplace_back(f, b, e);
  }
  for (auto& x : th) x.join();
}

// E in the split form the device uses: the element map (E-vector row -> true dof, or ntrue + c
// for the c-th row that is not a single weight 1), the rows C of those, and C^T over the true
// dofs it touches.  False if ntrue + nc passes 2^31 - 1.
struct HostE {
  int64_t nnz = 0, nc = 0;
  std::vector<int32_t> map;
  std::vector<int64_t> cptr;
  std::vector<int32_t> ccol;
  std::vector<double> cval;
  std::vector<int32_t> trow;
  std::vector<int64_t> tptr;
  std::vector<int32_t> tcol;
  std::vector<double> tval;
};

bool build_host_E(const Topo& T, const std::vector<int64_t>& order_elems,
                  const std::vector<int64_t>& first, int64_t nlocal, HostE& H) {
  // Rows of E: a single weight 1 goes into the element map; the others become rows of C.
  std::vector<int64_t> map(nlocal);
  std::vector<uint8_t> rown(nlocal);
  auto classify = [&](int64_t b, int64_t e_end) {
    Row r;
    for (int64_t t = b; t < e_end; ++t) {
      const int64_t e = order_elems[t];
      const int D = T.ord[e] + 1;
      for (int a = 0; a < D * D * D; ++a) {
        T.node_row(e, a % D, (a / D) % D, a / (D * D), r);
        const int64_t row = first[e] + a;
        rown[row] = (uint8_t)r.n;
        map[row] = (r.n == 1 && r.w[0] == 1.0) ? r.col[0] : -1;
      }
    }
  };
  parallel_for((int64_t)order_elems.size(), classify);
  int64_t nnz = 0, nc = 0;
  std::vector<int64_t> cptr(1, 0);
  for (int64_t row = 0; row < nlocal; ++row) {
    nnz += rown[row];
    if (map[row] < 0) {
      map[row] = T.ntrue + nc++;
      cptr.push_back(cptr.back() + rown[row]);
    }
  }
  if (T.ntrue + nc > 2147483647LL) return false;
  const int64_t cnnz = cptr.back();
  std::vector<int32_t> ccol(cnnz);
  std::vector<double> cval(cnnz);
  auto fill = [&](int64_t b, int64_t e_end) {
    Row r;
    for (int64_t t = b; t < e_end; ++t) {
      const int64_t e = order_elems[t];
      const int D = T.ord[e] + 1;
      for (int a = 0; a < D * D * D; ++a) {
        const int64_t row = first[e] + a;
        if (map[row] < T.ntrue) continue;
        T.node_row(e, a % D, (a / D) % D, a / (D * D), r);
        // columns ascending within a row (a fixed summation order): insertion sort
        for (int z = 1; z < r.n; ++z)
          for (int y = z; y > 0 && r.col[y - 1] > r.col[y]; --y) {
            std::swap(r.col[y - 1], r.col[y]);
            std::swap(r.w[y - 1], r.w[y]);
          }
        const int64_t o = cptr[map[row] - T.ntrue];
        for (int z = 0; z < r.n; ++z) {
          ccol[o + z] = (int32_t)r.col[z];
          cval[o + z] = r.w[z];
        }
      }
    }
  };
  parallel_for((int64_t)order_elems.size(), fill);
  std::vector<int32_t> map32(map.begin(), map.end());
  std::vector<int64_t>().swap(map);

  // C^T over the true dofs it touches (ascending), constrained rows ascending within each
  std::vector<int32_t> tcount(T.ntrue, 0);
  for (int64_t t = 0; t < cnnz; ++t) ++tcount[ccol[t]];
  std::vector<int32_t> trow;
  std::vector<int64_t> tptr(1, 0);
  std::vector<int64_t> tpos(T.ntrue, -1);
  for (int64_t i = 0; i < T.ntrue; ++i)
    if (tcount[i] > 0) {
      tpos[i] = tptr.back();
      trow.push_back((int32_t)i);
      tptr.push_back(tptr.back() + tcount[i]);
    }
  std::vector<int32_t> tcol(cnnz);
  std::vector<double> tval(cnnz);
  for (int64_t c = 0; c < nc; ++c)
    for (int64_t t = cptr[c]; t < cptr[c + 1]; ++t) {
      const int64_t o = tpos[ccol[t]]++;
      tcol[o] = (int32_t)c;
      tval[o] = cval[t];
    }

  H.nnz = nnz;
  H.nc = nc;
  H.map.swap(map32);
  H.cptr.swap(cptr);
  H.ccol.swap(ccol);
  H.cval.swap(cval);
  H.trow.swap(trow);
  H.tptr.swap(tptr);
  H.tcol.swap(tcol);
  H.tval.swap(tval);
  return true;
}

// 1 for the true dofs on the boundary of the box (vertices, edges and faces on it).
std::vector<uint8_t> boundary_mask(const Topo& T) {
  const int nx = T.n[0], ny = T.n[1], nz = T.n[2];
  std::vector<uint8_t> mask(T.ntrue, 0);
  {
    int64_t i[3];
    for (i[2] = 0; i[2] <= nz; ++i[2])
      for (i[1] = 0; i[1] <= ny; ++i[1])
        for (i[0] = 0; i[0] <= nx; ++i[0])
          mask[T.vertex(i)] = i[0] == 0 || i[1] == 0 || i[2] == 0 || i[0] == nx || i[1] == ny ||
                              i[2] == nz;
    for (int d = 0; d < 3; ++d) {
      for (i[2] = 0; i[2] < T.ebox[d][2]; ++i[2])
        for (i[1] = 0; i[1] < T.ebox[d][1]; ++i[1])
          for (i[0] = 0; i[0] < T.ebox[d][0]; ++i[0]) {
            const int64_t l = T.lin(T.ebox[d], i);
            if (T.on_boundary_edge(d, i))
              for (int m = 0; m < T.eq[d][l] - 1; ++m) mask[T.efirst[d][l] + m] = 1;
          }
      for (i[2] = 0; i[2] < T.fbox[d][2]; ++i[2])
        for (i[1] = 0; i[1] < T.fbox[d][1]; ++i[1])
          for (i[0] = 0; i[0] < T.fbox[d][0]; ++i[0]) {
            const int64_t l = T.lin(T.fbox[d], i);
            if (i[d] == 0 || i[d] == T.n[d])
              for (int m = 0; m < (T.fq[d][l] - 1) * (T.fq[d][l] - 1); ++m)
                mask[T.ffirst[d][l] + m] = 1;
          }
    }
  }

  return mask;
}

// E-vector layout: groups of ascending order, elements ascending within a group.  Returns the
// total length; first[e] the offset of element e, order_elems the elements in E-vector order.
int64_t evector_layout(const Topo& T, std::vector<int64_t>& first,
                       std::vector<int64_t>& order_elems) {
  first.assign(T.ne, 0);
  order_elems.clear();
  order_elems.reserve(T.ne);
  int present[kMaxOrder + 1] = {0};
  for (int p : T.ord) present[p] = 1;
  int64_t nlocal = 0;
  for (int p = 1; p <= kMaxOrder; ++p) {
    if (!present[p]) continue;
    for (int64_t e = 0; e < T.ne; ++e)
      if (T.ord[e] == p) {
        first[e] = nlocal;
        nlocal += (int64_t)(p + 1) * (p + 1) * (p + 1);
        order_elems.push_back(e);
      }
  }
  return nlocal;
}

__global__ void k_csr_gather(const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                             const double* __restrict__ val, int64_t nrows,
                             const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nrows;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = ptr[r], e = ptr[r + 1];
    double s = 0.0;
    for (int64_t t = b; t < e; ++t) s = fma(val[t], x[col[t]], s);
    y[r] = s;
  }
}

// ---- Jacobi-PCG on the variable-order space (same conventions as fe_pcg: x = 0 start,
// homogeneous essential conditions on the boundary mask, FP64 vectors, fixed-order reductions)

// dinv = 1/d on the free dofs, 0 on the boundary; flags[0] = 1 on a non-positive entry
__global__ void k_vs_dinv(const double* __restrict__ d, const uint8_t* __restrict__ mask,
                          double* __restrict__ dinv, int64_t n, int* flags) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (mask[i]) {
      dinv[i] = 0.0;
    } else {
      const double v = d[i];
      if (!(v > 0.0)) flags[0] = 1;
      dinv[i] = v > 0.0 ? 1.0 / v : 0.0;
    }
  }
}

// x = 0, r = (1-m) b, z = dinv r, p = z; partials r.z and b.b (free dofs)
__global__ void __launch_bounds__(kReduceThreads) k_vs_init(
    const double* __restrict__ b, const uint8_t* __restrict__ mask,
    const double* __restrict__ dinv, double* __restrict__ x, double* __restrict__ r,
    double* __restrict__ z, double* __restrict__ p, int64_t n, double* part0, double* part1) {
  double rz = 0.0, bb = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double bi = mask[i] ? 0.0 : b[i];
    const double zi = dinv[i] * bi;
    x[i] = 0.0;
    r[i] = bi;
    z[i] = zi;
    p[i] = zi;
    rz = fma(bi, zi, rz);
    bb = fma(bi, bi, bb);
  }
  block_sum2(rz, bb, part0, part1);
}

// partials of p.q over the free dofs (p is 0 on the boundary, so this is p.(1-m)Ap)
__global__ void __launch_bounds__(kReduceThreads) k_vs_pq(const double* __restrict__ p,
                                                          const double* __restrict__ q,
                                                          const uint8_t* __restrict__ mask,
                                                          int64_t n, double* part0) {
  double a = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (!mask[i]) a = fma(p[i], q[i], a);
  block_sum2(a, 0.0, part0, nullptr);
}

// x += alpha p, r -= alpha (1-m) q, z = dinv r; partials r.z and r.r
__global__ void __launch_bounds__(kReduceThreads) k_vs_update(
    double* __restrict__ x, double* __restrict__ r, double* __restrict__ z,
    const double* __restrict__ p, const double* __restrict__ q, const uint8_t* __restrict__ mask,
    const double* __restrict__ dinv, int64_t n, const double* __restrict__ sc, double* part0,
    double* part1) {
  const double alpha = sc[S_ALPHA];
  double rz = 0.0, rr = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = mask[i] ? r[i] : fma(-alpha, q[i], r[i]);
    const double zi = dinv[i] * ri;
    r[i] = ri;
    z[i] = zi;
    rz = fma(ri, zi, rz);
    rr = fma(ri, ri, rr);
  }
  block_sum2(rz, rr, part0, part1);
}

__global__ void k_vs_p(double* __restrict__ p, const double* __restrict__ z, int64_t n,
                       const double* __restrict__ sc) {
  const double beta = sc[S_BETA];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = fma(beta, p[i], z[i]);
}

// partials of ||(1-m)(b - q)||^2
__global__ void __launch_bounds__(kReduceThreads) k_vs_resid(const double* __restrict__ b,
                                                             const double* __restrict__ q,
                                                             const uint8_t* __restrict__ mask,
                                                             int64_t n, double* part0) {
  double a = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = mask[i] ? 0.0 : b[i] - q[i];
    a = fma(ri, ri, a);
  }
  block_sum2(a, 0.0, part0, nullptr);
}

// mode 0: rz, bb; 1: pq, alpha = rz / pq; 2: beta = rz' / rz, rz = rz', rr; 3: true residual
__global__ void __launch_bounds__(kFinishThreads) k_vs_finish(const double* part0,
                                                              const double* part1, double* sc,
                                                              int mode) {
  const double a = ordered_sum(part0);
  const double b = (mode == 0 || mode == 2) ? ordered_sum(part1) : 0.0;
  if (threadIdx.x != 0) return;
  if (mode == 0) {
    sc[S_RZ] = a;
    sc[S_BB] = b;
    sc[S_RR] = b;
  } else if (mode == 1) {
    sc[S_PQ] = a;
    sc[S_ALPHA] = sc[S_RZ] / a;
  } else if (mode == 2) {
    sc[S_BETA] = a / sc[S_RZ];
    sc[S_RZ] = a;
    sc[S_RR] = b;
  } else {
    sc[S_TRUE] = a;
  }
}

// e[t] = X[map[t]]: the E-vector from X = [x; C x] through the element map
__global__ void k_map_gather(const int32_t* __restrict__ map, int64_t n,
                             const double* __restrict__ X, double* __restrict__ e) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    e[t] = X[map[t]];
}

// y[rows[r]] += sum_t w_t Yc[col_t] (w_t = val_t, or val_t^2 with `square`): the transpose of the
// constrained rows over the true dofs they touch (distinct rows: no atomics, fixed order)
__global__ void k_ct_scatter(const int32_t* __restrict__ rows, const int64_t* __restrict__ ptr,
                             const int32_t* __restrict__ col, const double* __restrict__ val,
                             int64_t nrows, const double* __restrict__ Yc, double* __restrict__ y,
                             int square) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nrows;
       r += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t t = ptr[r]; t < ptr[r + 1]; ++t) {
      const double w = square ? val[t] * val[t] : val[t];
      s = fma(w, Yc[col[t]], s);
    }
    y[rows[r]] += s;
  }
}

unsigned grid_of(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16));
}

}  // namespace

// Most rows of E are a single weight 1 (a node that is itself a true dof): those stay in the
// element map, which points into X = [x; C x] with C the other ("constrained") rows of E, so the
// per-order kernels gather and scatter the true-dof vector directly; only C and its transpose
// need a sparse pass.
struct fe_vspace {
  int nx = 0, ny = 0, nz = 0, ops = 0;
  int64_t ne = 0, ntrue = 0, nlocal = 0, nnz = 0;
  int64_t nc = 0, cnnz = 0, nct = 0;    // constrained rows of E, their nonzeros, true dofs touched
  std::vector<int64_t> elem_first;      // [ne] E-vector offset per element
  double* d_vertices = nullptr;
  int32_t* d_map = nullptr;             // [nlocal] E-vector row -> index into X = [x; C x]
  int64_t* d_cptr = nullptr;            // C: [nc + 1]
  int32_t* d_ccol = nullptr;            //    true dof
  double* d_cval = nullptr;
  int32_t* d_trow = nullptr;            // C^T: [nct] true dof of each row
  int64_t* d_tptr = nullptr;            //      [nct + 1]
  int32_t* d_tcol = nullptr;            //      constrained row
  double* d_tval = nullptr;
  uint8_t* d_mask = nullptr;            // [ntrue]
  double* d_X = nullptr;                // [ntrue + nc]: x then C x
  double* d_Y = nullptr;                // [ntrue + nc]: the per-order kernels' scatter target
  int* d_zero = nullptr;                // a device 0: "y is zeroed by the caller" for the applies
  int* d_counter = nullptr;             // work counter of the persistent multi-order apply
  bool persistent = true;               // one persistent launch over all orders (else one each)
  double* d_Xb = nullptr;               // batched work vectors: [xb_cap][ntrue + nc] each
  double* d_Yb = nullptr;
  int xb_cap = 0;
  double* d_work = nullptr;             // PCG: x-free work vectors r, z, p, q, dinv [5][ntrue]
  double* d_red = nullptr;              //      2 kReduceBlocks partials + kScalars
  int* d_flags = nullptr;
  int ngroups = 0;
  int group_p[kMaxOrder];
  int64_t group_off[kMaxOrder];         // first E-vector row of the group
  fe_mesh* group_mesh[kMaxOrder];
  fe_pa* group_pa[kMaxOrder];
  // learned patch preconditioner: one network per order group (copies of networks trained on
  // single-order meshes), applied in the X numbering with one shared input/output scaling
  uint8_t* d_maskX = nullptr;           // [ntrue + nc]: rows of X without patch unknowns (the
                                        // boundary true dofs and every constrained row)
  fe_lpc* group_lpc[kMaxOrder] = {};    // owned
  int lpc_op = 0;
  double* d_FX = nullptr;               // [ntrue + nc]: the shared scaling (mult_X diag_X)^(-1/2)
  double* d_rm = nullptr;               // [ntrue]: the preconditioner's masked input
};

namespace {

void vspace_free(fe_vspace* vs) {
  for (int g = 0; g < vs->ngroups; ++g) {
    fe_lpc_destroy(vs->group_lpc[g]);
    fe_pa_destroy(vs->group_pa[g]);
    if (vs->group_mesh[g]) {
      vs->group_mesh[g]->d_vertices = nullptr;  // shared, freed below
      vs->group_mesh[g]->d_map = nullptr;       // a slice of vs->d_map
      vs->group_mesh[g]->d_mask = nullptr;      // vs->d_maskX, freed below
      fe_mesh_destroy(vs->group_mesh[g]);
    }
  }
  cudaFree(vs->d_vertices);
  cudaFree(vs->d_map);
  cudaFree(vs->d_cptr);
  cudaFree(vs->d_ccol);
  cudaFree(vs->d_cval);
  cudaFree(vs->d_trow);
  cudaFree(vs->d_tptr);
  cudaFree(vs->d_tcol);
  cudaFree(vs->d_tval);
  cudaFree(vs->d_mask);
  cudaFree(vs->d_maskX);
  cudaFree(vs->d_FX);
  cudaFree(vs->d_rm);
  cudaFree(vs->d_X);
  cudaFree(vs->d_Y);
  cudaFree(vs->d_zero);
  cudaFree(vs->d_counter);
  cudaFree(vs->d_Xb);
  cudaFree(vs->d_Yb);
  cudaFree(vs->d_work);
  cudaFree(vs->d_red);
  cudaFree(vs->d_flags);
  delete vs;
}

template <class T>
cudaError_t upload(T** dst, const std::vector<T>& src) {
  cudaError_t err = cudaMalloc(dst, sizeof(T) * std::max<size_t>(1, src.size()));
  if (err != cudaSuccess) return err;
  return cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice);
}

// X = [x; C x] on s (X: a work vector of ntrue + nc values; default the handle's)
int fill_X(const fe_vspace* vs, const double* x, cudaStream_t s, double* X = nullptr) {
  if (!X) X = vs->d_X;
  cudaError_t err = cudaMemcpyAsync(X, x, sizeof(double) * vs->ntrue,
                                    cudaMemcpyDeviceToDevice, s);
  if (err != cudaSuccess) return cuda_error(err, "fe_vspace: copy x");
  if (vs->nc > 0)
    k_csr_gather<<<grid_of(vs->nc), 256, 0, s>>>(vs->d_cptr, vs->d_ccol, vs->d_cval, vs->nc, x,
                                                 X + vs->ntrue);
  return cuda_error(cudaGetLastError(), "fe_vspace: constrained rows");
}

// y = Y[0, ntrue) + C^T Y[ntrue, ntrue + nc) (squared weights with `square`) on s
int fold_Y(const fe_vspace* vs, double* y, int square, cudaStream_t s, const double* Y = nullptr) {
  if (!Y) Y = vs->d_Y;
  cudaError_t err = cudaMemcpyAsync(y, Y, sizeof(double) * vs->ntrue,
                                    cudaMemcpyDeviceToDevice, s);
  if (err != cudaSuccess) return cuda_error(err, "fe_vspace: copy y");
  if (vs->nct > 0)
    k_ct_scatter<<<grid_of(vs->nct), 256, 0, s>>>(vs->d_trow, vs->d_tptr, vs->d_tcol, vs->d_tval,
                                                  vs->nct, Y + vs->ntrue, y, square);
  return cuda_error(cudaGetLastError(), "fe_vspace: constrained transpose");
}

}  // namespace

extern "C" {

static int vspace_setup(int nx, int ny, int nz, const int32_t* host_order,
                        const double* host_vertices, const double* host_coeff, int ops,
                        void* stream, fe_vspace** out) {
  if (!out) return set_error(FE_ERR_ARG, "fe_vspace_setup: out is NULL");
  *out = nullptr;
  if (!host_order || !host_vertices) return set_error(FE_ERR_ARG, "fe_vspace_setup: null argument");
  if (nx < 1 || ny < 1 || nz < 1) return set_error(FE_ERR_ARG, "fe_vspace_setup: mesh size < 1");
  if (ops <= 0 || (ops & ~(FE_DIFFUSION | FE_MASS)))
    return set_error(FE_ERR_ARG, "fe_vspace_setup: ops must be FE_DIFFUSION and/or FE_MASS");
  Topo T;
  if (!build_topology(nx, ny, nz, host_order, T))
    return set_error(FE_ERR_ARG, "fe_vspace_setup: orders must be 1..8");
  cudaStream_t s = (cudaStream_t)stream;

  std::vector<int64_t> first, order_elems;
  const int64_t nlocal = evector_layout(T, first, order_elems);
  int present[kMaxOrder + 1] = {0};
  for (int p : T.ord) present[p] = 1;
  if (T.ntrue > 2147483647LL || nlocal > 2147483647LL)
    return set_error(FE_ERR_UNSUPPORTED, "fe_vspace_setup: more than 2^31-1 true or local dofs");

  HostE H;
  if (!build_host_E(T, order_elems, first, nlocal, H))
    return set_error(FE_ERR_UNSUPPORTED, "fe_vspace_setup: more than 2^31-1 constrained values");
  const int64_t nnz = H.nnz, nc = H.nc;

  std::vector<uint8_t> mask = boundary_mask(T);

  fe_vspace* vs = new fe_vspace();
  vs->nx = nx;
  vs->ny = ny;
  vs->nz = nz;
  vs->ops = ops;
  vs->ne = T.ne;
  vs->ntrue = T.ntrue;
  vs->nlocal = nlocal;
  vs->nnz = nnz;
  vs->nc = nc;
  vs->nct = (int64_t)H.trow.size();
  vs->cnnz = H.cptr.back();
  vs->elem_first = first;
  const int64_t nv = T.nv, nX = T.ntrue + nc;
  cudaError_t err = cudaMalloc(&vs->d_vertices, sizeof(double) * 3 * nv);
  if (err == cudaSuccess)
    err = cudaMemcpy(vs->d_vertices, host_vertices, sizeof(double) * 3 * nv, cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = upload(&vs->d_map, H.map);
  if (err == cudaSuccess) err = upload(&vs->d_cptr, H.cptr);
  if (err == cudaSuccess) err = upload(&vs->d_ccol, H.ccol);
  if (err == cudaSuccess) err = upload(&vs->d_cval, H.cval);
  if (err == cudaSuccess) err = upload(&vs->d_trow, H.trow);
  if (err == cudaSuccess) err = upload(&vs->d_tptr, H.tptr);
  if (err == cudaSuccess) err = upload(&vs->d_tcol, H.tcol);
  if (err == cudaSuccess) err = upload(&vs->d_tval, H.tval);
  if (err == cudaSuccess) err = upload(&vs->d_mask, mask);
  if (err == cudaSuccess) {
    // X rows without patch unknowns: the boundary true dofs, and every constrained row (its
    // value interpolates true dofs that are patch unknowns of the elements owning them, so
    // gathering the residual there as well would count it twice)
    std::vector<uint8_t> maskX(mask.begin(), mask.end());
    maskX.resize((size_t)nX, 1);
    err = upload(&vs->d_maskX, maskX);
  }
  if (err == cudaSuccess) err = cudaMalloc(&vs->d_X, sizeof(double) * std::max<int64_t>(1, nX));
  if (err == cudaSuccess) err = cudaMalloc(&vs->d_Y, sizeof(double) * std::max<int64_t>(1, nX));
  if (err == cudaSuccess) err = cudaMalloc(&vs->d_zero, sizeof(int));
  if (err == cudaSuccess) err = cudaMemset(vs->d_zero, 0, sizeof(int));
  if (err == cudaSuccess) err = cudaMalloc(&vs->d_counter, sizeof(int));
  if (err != cudaSuccess) {
    vspace_free(vs);
    return cuda_error(err, "fe_vspace_setup: upload");
  }

  // one partial assembly per order present, over that order's elements; each group's element
  // map is its slice of d_map, into X / Y of length ntrue + nc
  int64_t t0 = 0;
  for (int p = 1; p <= kMaxOrder; ++p) {
    if (!present[p]) continue;
    const int g = vs->ngroups++;
    vs->group_p[g] = p;
    vs->group_mesh[g] = nullptr;
    vs->group_pa[g] = nullptr;
    std::vector<int32_t> ids;
    std::vector<double> coeff;
    while (t0 < (int64_t)order_elems.size() && T.ord[order_elems[t0]] == p) {
      ids.push_back((int32_t)order_elems[t0]);
      if (host_coeff) coeff.push_back(host_coeff[order_elems[t0]]);
      ++t0;
    }
    vs->group_off[g] = first[ids[0]];
    fe_mesh* m = new fe_mesh();
    vs->group_mesh[g] = m;
    m->nx = nx;
    m->ny = ny;
    m->nz = nz;
    m->p = p;
    m->D = p + 1;
    m->ne = (int64_t)ids.size();
    m->ndofs = nX;
    cudaGetDevice(&m->device);
    m->d_vertices = vs->d_vertices;
    m->d_map = vs->d_map + vs->group_off[g];
    m->d_mask = vs->d_maskX;
    err = upload(&m->d_elem_ids, ids);
    double* dc = nullptr;
    if (err == cudaSuccess && host_coeff) err = upload(&dc, coeff);
    if (err != cudaSuccess) {
      cudaFree(dc);
      vspace_free(vs);
      return cuda_error(err, "fe_vspace_setup: order group");
    }
    const int st = fe_pa_setup(m, 0, dc, ops, stream, &vs->group_pa[g]);
    cudaFree(dc);
    if (st != FE_OK) {
      const std::string msg = fe_last_error();
      vspace_free(vs);
      return set_error(st, "fe_vspace_setup: " + msg);
    }
  }
  err = cudaStreamSynchronize(s);
  if (err != cudaSuccess) {
    vspace_free(vs);
    return cuda_error(err, "fe_vspace_setup");
  }
  *out = vs;
  return FE_OK;
}

static int vspace_host_E(int nx, int ny, int nz, const int32_t* host_order, int64_t* ntrue,
                         int64_t* nlocal, int64_t* nnz, int64_t* rowptr, int32_t* cols,
                         double* vals, int64_t* elem_first, uint8_t* mask) {
  if (!host_order || !ntrue || !nlocal || !nnz)
    return set_error(FE_ERR_ARG, "fe_vspace_host_E: null argument");
  if (nx < 1 || ny < 1 || nz < 1) return set_error(FE_ERR_ARG, "fe_vspace_host_E: mesh size < 1");
  Topo T;
  if (!build_topology(nx, ny, nz, host_order, T))
    return set_error(FE_ERR_ARG, "fe_vspace_host_E: orders must be 1..8");
  std::vector<int64_t> first, order_elems;
  const int64_t nl = evector_layout(T, first, order_elems);
  std::vector<int64_t> cnt(nl + 1, 0);
  auto count = [&](int64_t b, int64_t e_end) {
    Row r;
    for (int64_t t = b; t < e_end; ++t) {
      const int64_t e = order_elems[t];
      const int D = T.ord[e] + 1;
      for (int a = 0; a < D * D * D; ++a) {
        T.node_row(e, a % D, (a / D) % D, a / (D * D), r);
        cnt[first[e] + a + 1] = r.n;
      }
    }
  };
  parallel_for((int64_t)order_elems.size(), count);
  for (int64_t r = 0; r < nl; ++r) cnt[r + 1] += cnt[r];
  *ntrue = T.ntrue;
  *nlocal = nl;
  *nnz = cnt[nl];
  if (rowptr) std::memcpy(rowptr, cnt.data(), sizeof(int64_t) * (nl + 1));
  if (elem_first) std::memcpy(elem_first, first.data(), sizeof(int64_t) * T.ne);
  if (mask) {
    const std::vector<uint8_t> m = boundary_mask(T);
    std::memcpy(mask, m.data(), (size_t)T.ntrue);
  }
  if (cols && vals) {
    auto fill = [&](int64_t b, int64_t e_end) {
      Row r;
      for (int64_t t = b; t < e_end; ++t) {
        const int64_t e = order_elems[t];
        const int D = T.ord[e] + 1;
        for (int a = 0; a < D * D * D; ++a) {
          T.node_row(e, a % D, (a / D) % D, a / (D * D), r);
          const int64_t o = cnt[first[e] + a];
          for (int z = 0; z < r.n; ++z) {
            cols[o + z] = (int32_t)r.col[z];
            vals[o + z] = r.w[z];
          }
        }
      }
    };
    parallel_for((int64_t)order_elems.size(), fill);
  }
  return FE_OK;
}

// The host construction allocates large vectors and starts threads: a failure there becomes a
// status code instead of an exception crossing the C ABI.
int fe_vspace_setup(int nx, int ny, int nz, const int32_t* host_order,
                    const double* host_vertices, const double* host_coeff, int ops, void* stream,
                    fe_vspace** out) {
  clear_error();
  try {
    return vspace_setup(nx, ny, nz, host_order, host_vertices, host_coeff, ops, stream, out);
  } catch (const std::bad_alloc&) {
    return set_error(FE_ERR_OOM, "fe_vspace_setup: host allocation failed");
  } catch (const std::exception& e) {
    return set_error(FE_ERR_CUDA, std::string("fe_vspace_setup: ") + e.what());
  }
}

int fe_vspace_host_E(int nx, int ny, int nz, const int32_t* host_order, int64_t* ntrue,
                     int64_t* nlocal, int64_t* nnz, int64_t* rowptr, int32_t* cols, double* vals,
                     int64_t* elem_first, uint8_t* mask) {
  clear_error();
  try {
    return vspace_host_E(nx, ny, nz, host_order, ntrue, nlocal, nnz, rowptr, cols, vals,
                         elem_first, mask);
  } catch (const std::bad_alloc&) {
    return set_error(FE_ERR_OOM, "fe_vspace_host_E: host allocation failed");
  } catch (const std::exception& e) {
    return set_error(FE_ERR_ARG, std::string("fe_vspace_host_E: ") + e.what());
  }
}

int fe_vspace_sizes(const fe_vspace* vs, int64_t* ntrue, int64_t* nlocal, int64_t* nnz) {
  clear_error();
  if (!vs) return set_error(FE_ERR_ARG, "fe_vspace_sizes: handle is NULL");
  if (ntrue) *ntrue = vs->ntrue;
  if (nlocal) *nlocal = vs->nlocal;
  if (nnz) *nnz = vs->nnz;
  return FE_OK;
}

int fe_vspace_constraint_sizes(const fe_vspace* vs, int64_t* nrows, int64_t* nnz,
                               int64_t* ntouched) {
  clear_error();
  if (!vs) return set_error(FE_ERR_ARG, "fe_vspace_constraint_sizes: handle is NULL");
  if (nrows) *nrows = vs->nc;
  if (nnz) *nnz = vs->cnnz;
  if (ntouched) *ntouched = vs->nct;
  return FE_OK;
}

int fe_vspace_layout(const fe_vspace* vs, int64_t* host_first) {
  clear_error();
  if (!vs || !host_first) return set_error(FE_ERR_ARG, "fe_vspace_layout: null argument");
  std::memcpy(host_first, vs->elem_first.data(), sizeof(int64_t) * vs->ne);
  return FE_OK;
}

int fe_vspace_boundary_mask(const fe_vspace* vs, uint8_t* dev_mask, void* stream) {
  clear_error();
  if (!vs || !dev_mask) return set_error(FE_ERR_ARG, "fe_vspace_boundary_mask: null argument");
  cudaError_t err = cudaMemcpyAsync(dev_mask, vs->d_mask, (size_t)vs->ntrue,
                                    cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
  if (err != cudaSuccess) return cuda_error(err, "fe_vspace_boundary_mask");
  return FE_OK;
}

int fe_vspace_set_variant(fe_vspace* vs, int variant, void* stream) {
  clear_error();
  if (!vs) return set_error(FE_ERR_ARG, "fe_vspace_set_variant: handle is NULL");
  for (int g = 0; g < vs->ngroups; ++g) {
    const int st = fe_pa_set_variant(vs->group_pa[g], variant, stream);
    if (st != FE_OK) return st;
  }
  return FE_OK;
}

int fe_vspace_set_persistent(fe_vspace* vs, int enable) {
  clear_error();
  if (!vs) return set_error(FE_ERR_ARG, "fe_vspace_set_persistent: handle is NULL");
  vs->persistent = enable != 0;
  return FE_OK;
}

int fe_vspace_prolong(const fe_vspace* vs, const double* dev_x, double* dev_e, void* stream) {
  clear_error();
  if (!vs || !dev_x || !dev_e) return set_error(FE_ERR_ARG, "fe_vspace_prolong: null argument");
  cudaStream_t s = (cudaStream_t)stream;
  const int st = fill_X(vs, dev_x, s);
  if (st != FE_OK) return st;
  k_map_gather<<<grid_of(vs->nlocal), 256, 0, s>>>(vs->d_map, vs->nlocal, vs->d_X, dev_e);
  return cuda_error(cudaGetLastError(), "fe_vspace_prolong: launch");
}

}  // extern "C"

namespace {
// The order groups of vs for the persistent multi-order apply with `variant`, highest order
// first (its items are the largest); false if that apply is not built for the variant.
bool multi_groups(const fe_vspace* vs, int op, int variant, MultiGroups* g,
                  const Basis1D** basis) {
  if (variant != FE_VARIANT_F64 && variant != FE_VARIANT_F32X2) return false;
  for (int p = 0; p < kMaxOrder; ++p) basis[p] = nullptr;
  g->n = 0;
  g->first_item[0] = 0;
  for (int k = vs->ngroups - 1; k >= 0; --k) {
    const fe_pa* pa = vs->group_pa[k];
    const int p = vs->group_p[k];
    const int ne_item = multi_elems(variant, op, p);
    if (ne_item <= 0) return false;
    const int i = g->n++;
    g->order[i] = p;
    g->map[i] = pa->mesh->d_map;
    g->ne[i] = pa->mesh->ne;
    if (variant == FE_VARIANT_F32X2) {
      g->qd[i] = op == FE_DIFFUSION ? pa->d_qd_diff2 : pa->d_qd_mass2;
      g->qscale[i] = op == FE_DIFFUSION ? pa->d_qs_diff : pa->d_qs_mass;
      if (!g->qd[i] || !g->qscale[i]) return false;
    } else {
      g->qd[i] = op == FE_DIFFUSION ? pa->d_qd_diff : pa->d_qd_mass;
      g->qscale[i] = nullptr;
    }
    g->first_item[i + 1] = g->first_item[i] + (g->ne[i] + ne_item - 1) / ne_item;
    basis[p - 1] = &pa->basis;
  }
  return true;
}

// y_r = E^T blockdiag(A_e) E x_r for r < nrhs (x_r = x + r ldx, y_r = y + r ldy) with the given
// variant (-1: each order's selected variant), through the work vectors X, Y of nrhs (ntrue + nc)
// values: one persistent launch over all orders and right-hand sides when every group uses the
// same FP64-accurate arithmetic (and persistent launches are on), else one fused launch per
// order.  nk (optional) counts the kernels.
int vspace_apply_b(const fe_vspace* vs, int op, int variant, int nrhs, const double* dev_x,
                   int64_t ldx, double* dev_y, int64_t ldy, double* X, double* Y,
                   cudaStream_t s, int* nk = nullptr) {
  const int64_t nX = vs->ntrue + vs->nc;
  int st;
  for (int r = 0; r < nrhs; ++r)
    if ((st = fill_X(vs, dev_x + r * ldx, s, X + r * nX)) != FE_OK) return st;
  cudaError_t err = cudaMemsetAsync(Y, 0, sizeof(double) * nX * nrhs, s);
  if (err != cudaSuccess) return cuda_error(err, "fe_vspace_apply: zero Y");
  if (nk) *nk += nrhs * (vs->nc > 0 ? 1 : 0);
  int v0 = variant < 0 ? vs->group_pa[0]->variant : variant;
  bool uniform = true;
  for (int g = 0; g < vs->ngroups; ++g)
    if ((variant < 0 ? vs->group_pa[g]->variant : variant) != v0) uniform = false;
  MultiGroups mg;
  const Basis1D* basis[kMaxOrder];
  if (vs->persistent && uniform && multi_groups(vs, op, v0, &mg, basis)) {
    if ((st = launch_apply_multi(v0, op, mg, basis, X, Y, vs->d_counter, nrhs, nX, nX, s)) !=
        FE_OK)
      return st;
    if (nk) *nk += 1;
  } else {
    for (int g = 0; g < vs->ngroups; ++g) {
      const fe_pa* pa = vs->group_pa[g];
      if ((st = apply_dispatch(pa, op, variant < 0 ? pa->variant : variant, X, Y, s, vs->d_zero,
                               nullptr, nullptr, false, nrhs, nX, nX)) != FE_OK)
        return st;
      if (nk) *nk += 1;
    }
  }
  for (int r = 0; r < nrhs; ++r)
    if ((st = fold_Y(vs, dev_y + r * ldy, 0, s, Y + r * nX)) != FE_OK) return st;
  if (nk) *nk += nrhs * (vs->nct > 0 ? 1 : 0);
  return FE_OK;
}

// the single right-hand side through the handle's work vectors
int vspace_apply(const fe_vspace* vs, int op, int variant, const double* dev_x, double* dev_y,
                 cudaStream_t s) {
  return vspace_apply_b(vs, op, variant, 1, dev_x, 0, dev_y, 0, vs->d_X, vs->d_Y, s);
}

}  // namespace

namespace fe {
int multi_elems(int variant, int op, int order) {
  if (variant == FE_VARIANT_F64) return multi_elems_f64(op, order);
  if (variant == FE_VARIANT_F32X2) return multi_elems_f32x2(op, order);
  return 0;
}
int launch_apply_multi(int variant, int op, const MultiGroups& g, const Basis1D* const* basis,
                       const double* x, double* y, int* counter, int nrhs, int64_t ldx,
                       int64_t ldy, cudaStream_t s) {
  if (variant == FE_VARIANT_F64)
    return launch_apply_multi_f64(op, g, basis, x, y, counter, nrhs, ldx, ldy, s);
  if (variant == FE_VARIANT_F32X2)
    return launch_apply_multi_f32x2(op, g, basis, x, y, counter, nrhs, ldx, ldy, s);
  return set_error(FE_ERR_UNSUPPORTED, "multi-order apply: variant not built");
}
}  // namespace fe

extern "C" {

int fe_vspace_apply(const fe_vspace* vs, int op, const double* dev_x, double* dev_y,
                    void* stream) {
  clear_error();
  if (!vs || !dev_x || !dev_y) return set_error(FE_ERR_ARG, "fe_vspace_apply: null argument");
  if (op != FE_DIFFUSION && op != FE_MASS) return set_error(FE_ERR_ARG, "fe_vspace_apply: bad op");
  if (!(vs->ops & op))
    return set_error(FE_ERR_ARG, "fe_vspace_apply: operator not set up in fe_vspace_setup");
  return vspace_apply(vs, op, -1, dev_x, dev_y, (cudaStream_t)stream);
}

int fe_vspace_diagonal(const fe_vspace* vs, int op, double* dev_diag, void* stream) {
  clear_error();
  if (!vs || !dev_diag) return set_error(FE_ERR_ARG, "fe_vspace_diagonal: null argument");
  if (op != FE_DIFFUSION && op != FE_MASS)
    return set_error(FE_ERR_ARG, "fe_vspace_diagonal: bad op");
  if (!(vs->ops & op))
    return set_error(FE_ERR_ARG, "fe_vspace_diagonal: operator not set up in fe_vspace_setup");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t err = cudaMemsetAsync(vs->d_Y, 0, sizeof(double) * (vs->ntrue + vs->nc), s);
  if (err != cudaSuccess) return cuda_error(err, "fe_vspace_diagonal: zero Y");
  for (int g = 0; g < vs->ngroups; ++g) {
    const int st = diagonal_accumulate(vs->group_pa[g], op, vs->d_Y, s);
    if (st != FE_OK) return st;
  }
  return fold_Y(vs, dev_diag, 1, s);
}

int fe_vspace_pcg(fe_vspace* vs, int op, const double* dev_b, double* dev_x, double rtol,
                  int maxit, fe_pcg_stats* stats, void* stream) {
  clear_error();
  const auto t0 = std::chrono::steady_clock::now();
  if (stats) *stats = fe_pcg_stats{0, 0.0, 0.0, 0.0, 0, 0};
  if (!vs || !dev_b || !dev_x) return set_error(FE_ERR_ARG, "fe_vspace_pcg: null argument");
  if (op != FE_DIFFUSION && op != FE_MASS) return set_error(FE_ERR_ARG, "fe_vspace_pcg: bad op");
  if (!(vs->ops & op)) return set_error(FE_ERR_ARG, "fe_vspace_pcg: operator not set up");
  if (maxit < 1 || !(rtol >= 0.0)) return set_error(FE_ERR_ARG, "fe_vspace_pcg: bad rtol or maxit");
  for (int g = 0; g < vs->ngroups; ++g)
    if (vs->group_pa[g]->variant == FE_VARIANT_F32)
      return set_error(FE_ERR_UNSUPPORTED, "fe_vspace_pcg: the FP32 variant is not FP64-accurate");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = vs->ntrue;
  cudaError_t err = cudaSuccess;
  if (!vs->d_work) {
    if ((err = cudaMalloc(&vs->d_work, sizeof(double) * 5 * n)) != cudaSuccess ||
        (err = cudaMalloc(&vs->d_red, sizeof(double) * (2 * kReduceBlocks + kScalars))) !=
            cudaSuccess ||
        (err = cudaMalloc(&vs->d_flags, sizeof(int) * 4)) != cudaSuccess) {
      cudaFree(vs->d_work);
      cudaFree(vs->d_red);
      vs->d_work = nullptr;
      vs->d_red = nullptr;
      return cuda_error(err, "fe_vspace_pcg: workspace cudaMalloc");
    }
  }
  double *r = vs->d_work, *z = r + n, *p = z + n, *q = p + n, *dinv = q + n;
  double *part0 = vs->d_red, *part1 = part0 + kReduceBlocks, *sc = part1 + kReduceBlocks;
  int launches = 0;
  // Jacobi: the diagonal of E^T diag(A_E) E (q as scratch), inverted on the free dofs
  int st = fe_vspace_diagonal(vs, op, q, stream);
  if (st != FE_OK) return st;
  cudaMemsetAsync(vs->d_flags, 0, sizeof(int) * 4, s);
  k_vs_dinv<<<grid_of(n), 256, 0, s>>>(q, vs->d_mask, dinv, n, vs->d_flags);
  k_vs_init<<<kReduceBlocks, kReduceThreads, 0, s>>>(dev_b, vs->d_mask, dinv, dev_x, r, z, p, n,
                                                     part0, part1);
  k_vs_finish<<<1, kFinishThreads, 0, s>>>(part0, part1, sc, 0);
  launches += 2 * vs->ngroups + 4;
  double hsc[kScalars];
  int hflag = 0;
  auto read_sc = [&]() -> int {
    cudaError_t e;
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(hsc, sc, sizeof(hsc), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
      return cuda_error(e, "fe_vspace_pcg: iteration");
    return FE_OK;
  };
  if ((st = read_sc()) != FE_OK) return st;
  if ((err = cudaMemcpy(&hflag, vs->d_flags, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_error(err, "fe_vspace_pcg: diagonal check");
  if (hflag) return set_error(FE_ERR_BREAKDOWN, "fe_vspace_pcg: non-positive diagonal entry");
  const double bb = hsc[S_BB];
  int status = FE_ERR_NOT_CONVERGED, iters = 0;
  double rel = bb > 0.0 ? 1.0 : 0.0;
  if (!(bb > 0.0)) status = std::isfinite(bb) ? FE_OK : FE_ERR_NAN;
  for (int it = 1; status == FE_ERR_NOT_CONVERGED && it <= maxit; ++it) {
    if ((st = fe_vspace_apply(vs, op, p, q, stream)) != FE_OK) return st;
    k_vs_pq<<<kReduceBlocks, kReduceThreads, 0, s>>>(p, q, vs->d_mask, n, part0);
    k_vs_finish<<<1, kFinishThreads, 0, s>>>(part0, part1, sc, 1);
    k_vs_update<<<kReduceBlocks, kReduceThreads, 0, s>>>(dev_x, r, z, p, q, vs->d_mask, dinv, n, sc,
                                                        part0, part1);
    k_vs_finish<<<1, kFinishThreads, 0, s>>>(part0, part1, sc, 2);
    launches += vs->ngroups + 6;
    if ((st = read_sc()) != FE_OK) return st;
    iters = it;
    rel = std::sqrt(hsc[S_RR] / bb);
    if (!std::isfinite(rel) || !std::isfinite(hsc[S_PQ])) {
      status = FE_ERR_NAN;
    } else if (!(hsc[S_PQ] > 0.0)) {
      status = FE_ERR_BREAKDOWN;
    } else if (rel <= rtol) {
      status = FE_OK;
    } else {
      k_vs_p<<<grid_of(n), 256, 0, s>>>(p, z, n, sc);
      ++launches;
    }
  }
  // true residual ||(1-m)(b - A x)|| / ||(1-m) b|| with the FP64 operator
  double true_rel = 0.0;
  if ((st = vspace_apply(vs, op, FE_VARIANT_F64, dev_x, q, s)) != FE_OK) return st;
  k_vs_resid<<<kReduceBlocks, kReduceThreads, 0, s>>>(dev_b, q, vs->d_mask, n, part0);
  k_vs_finish<<<1, kFinishThreads, 0, s>>>(part0, part1, sc, 3);
  launches += vs->ngroups + 4;
  if ((st = read_sc()) != FE_OK) return st;
  if (bb > 0.0) true_rel = std::sqrt(hsc[S_TRUE] / bb);
  if (stats) {
    stats->iters = iters;
    stats->rel_resid = rel;
    stats->true_rel_resid = true_rel;
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    stats->launches = launches;
    stats->outer_iters = 1;
  }
  switch (status) {
    case FE_OK:
      return FE_OK;
    case FE_ERR_BREAKDOWN:
      return set_error(FE_ERR_BREAKDOWN, "fe_vspace_pcg: p.Ap <= 0");
    case FE_ERR_NAN:
      return set_error(FE_ERR_NAN, "fe_vspace_pcg: NaN or Inf in the iteration");
    default:
      return set_error(FE_ERR_NOT_CONVERGED, "fe_vspace_pcg: maxit reached before rtol");
  }
}

}  // extern "C"

namespace {
// Batched work vectors for nrhs right-hand sides (kept with the handle, grown on demand).
int batched_work(const fe_vspace* cvs, int nrhs) {
  fe_vspace* vs = const_cast<fe_vspace*>(cvs);
  if (nrhs <= vs->xb_cap) return FE_OK;
  cudaFree(vs->d_Xb);
  cudaFree(vs->d_Yb);
  vs->d_Xb = vs->d_Yb = nullptr;
  vs->xb_cap = 0;
  const size_t bytes = sizeof(double) * (size_t)(vs->ntrue + vs->nc) * nrhs;
  cudaError_t err;
  if ((err = cudaMalloc(&vs->d_Xb, bytes)) != cudaSuccess ||
      (err = cudaMalloc(&vs->d_Yb, bytes)) != cudaSuccess)
    return cuda_error(err, "fe_vspace: batched work vectors");
  vs->xb_cap = nrhs;
  return FE_OK;
}
}  // namespace

extern "C" {

int fe_vspace_apply_batched(const fe_vspace* vs, int op, int nrhs, const double* dev_x,
                            int64_t ldx, double* dev_y, int64_t ldy, void* stream) {
  clear_error();
  if (!vs || !dev_x || !dev_y) return set_error(FE_ERR_ARG, "fe_vspace_apply_batched: null argument");
  if (op != FE_DIFFUSION && op != FE_MASS) return set_error(FE_ERR_ARG, "fe_vspace_apply_batched: bad op");
  if (!(vs->ops & op)) return set_error(FE_ERR_ARG, "fe_vspace_apply_batched: operator not set up");
  if (nrhs < 1 || nrhs > 1024 || ldx < vs->ntrue || ldy < vs->ntrue)
    return set_error(FE_ERR_ARG, "fe_vspace_apply_batched: need 1 <= nrhs <= 1024, ld >= ntrue");
  int st = batched_work(vs, nrhs);
  if (st != FE_OK) return st;
  return vspace_apply_b(vs, op, -1, nrhs, dev_x, ldx, dev_y, ldy, vs->d_Xb, vs->d_Yb,
                        (cudaStream_t)stream);
}

int fe_vspace_pcg_batched(fe_vspace* vs, int op, int nrhs, const double* dev_b, int64_t ldb,
                          double* dev_x, int64_t ldx, double rtol, int maxit,
                          fe_pcg_stats* stats, void* stream) {
  clear_error();
  if (!vs || !dev_b || !dev_x) return set_error(FE_ERR_ARG, "fe_vspace_pcg_batched: null argument");
  if (op != FE_DIFFUSION && op != FE_MASS) return set_error(FE_ERR_ARG, "fe_vspace_pcg_batched: bad op");
  if (!(vs->ops & op)) return set_error(FE_ERR_ARG, "fe_vspace_pcg_batched: operator not set up");
  for (int g = 0; g < vs->ngroups; ++g)
    if (vs->group_pa[g]->variant == FE_VARIANT_F32)
      return set_error(FE_ERR_UNSUPPORTED,
                       "fe_vspace_pcg_batched: the FP32 variant is not FP64-accurate");
  if (nrhs < 1 || nrhs > 1024) return set_error(FE_ERR_ARG, "fe_vspace_pcg_batched: bad nrhs");
  int st = batched_work(vs, nrhs);
  if (st != FE_OK) return st;
  const int64_t n = vs->ntrue;
  BatchedOperator A;
  A.n = n;
  A.mask = vs->d_mask;
  A.apply = [=](cudaStream_t q, int nr, const double* P, double* Q, const int*, int* nk) {
    return vspace_apply_b(vs, op, -1, nr, P, n, Q, n, vs->d_Xb, vs->d_Yb, q, nk);
  };
  A.apply_fp64 = [=](cudaStream_t q, int nr, const double* X, int64_t lx, double* Q, int* nk) {
    return vspace_apply_b(vs, op, FE_VARIANT_F64, nr, X, lx, Q, n, vs->d_Xb, vs->d_Yb, q, nk);
  };
  A.diagonal = [=](cudaStream_t q, double* d) { return fe_vspace_diagonal(vs, op, d, q); };
  return pcg_batched_core(A, nrhs, dev_b, ldb, dev_x, ldx, rtol, maxit, stats,
                          (cudaStream_t)stream, "fe_vspace_pcg_batched");
}

void fe_vspace_destroy(fe_vspace* vs) {
  if (vs) vspace_free(vs);
}

}  // extern "C"

// ---- the learned patch preconditioner on a variable-order space: M(r) = E^T F_X
//      sum_e R_e^T s_e f_p(e)(x_e / s_e), x_e = R_e F_X E r, one network f_p per order (the
//      order group's copy of a network trained on a single-order mesh), R_e the element's rows
//      of X = [r; C r], F_X the shared scaling (mult_X diag_X)^(-1/2) of the X rows: mult_X counts
//      the element rows of every order mapped to an X row, diag_X is the space's Jacobi diagonal
//      diag(E^T blockdiag(diag A_e) E) of its true dof (the higher-order neighbours reading it
//      through constrained nodes included), and F_X is 0 on the rows without patch unknowns (the
//      boundary true dofs and every constrained row).  With one order everywhere this is the
//      single-order operator.
namespace {

__global__ void k_count_rows(const int32_t* __restrict__ map, int64_t n, double* __restrict__ c) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&c[map[i]], 1.0);
}

__global__ void k_fx(const double* __restrict__ mult, const double* __restrict__ diag,
                     const uint8_t* __restrict__ mask, double* __restrict__ F, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double m = mult[i], d = diag[i];
    F[i] = (mask[i] || !(m > 0.0) || !(d > 0.0)) ? 0.0 : 1.0 / sqrt(m * d);
  }
}

__global__ void k_mask_copy(const double* __restrict__ r, const uint8_t* __restrict__ mask,
                            double* __restrict__ out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = mask[i] ? 0.0 : r[i];
}

__global__ void k_mask_zero(double* __restrict__ z, const uint8_t* __restrict__ mask, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (mask[i]) z[i] = 0.0;
}

// F_X for operator op, handed to every attached group network.
int vspace_lpc_scaling(fe_vspace* vs, int op, cudaStream_t s) {
  const int64_t nX = vs->ntrue + vs->nc;
  cudaError_t err = cudaSuccess;
  if (!vs->d_FX && (err = cudaMalloc(&vs->d_FX, sizeof(double) * nX)) != cudaSuccess) {
    vs->d_FX = nullptr;
    return cuda_error(err, "fe_vspace_set_learned: scaling cudaMalloc");
  }
  double* mult = nullptr;
  if ((err = cudaMalloc(&mult, sizeof(double) * (nX + vs->ntrue))) != cudaSuccess)
    return cuda_error(err, "fe_vspace_set_learned: scaling cudaMalloc");
  double* dtrue = mult + nX;
  int st = FE_OK;
  cudaMemsetAsync(mult, 0, sizeof(double) * nX, s);
  k_count_rows<<<grid_of(vs->nlocal), 256, 0, s>>>(vs->d_map, vs->nlocal, mult);
  cudaMemsetAsync(vs->d_Y, 0, sizeof(double) * nX, s);
  for (int g = 0; g < vs->ngroups && st == FE_OK; ++g)
    st = diagonal_accumulate(vs->group_pa[g], op, vs->d_Y, s);
  // the true-dof rows take the space's Jacobi diagonal (constrained rows folded in)
  if (st == FE_OK) st = fold_Y(vs, dtrue, 1, s);
  if (st == FE_OK)
    st = cuda_error(cudaMemcpyAsync(vs->d_Y, dtrue, sizeof(double) * vs->ntrue,
                                    cudaMemcpyDeviceToDevice, s),
                    "fe_vspace_set_learned: scaling copy");
  if (st == FE_OK) {
    k_fx<<<grid_of(nX), 256, 0, s>>>(mult, vs->d_Y, vs->d_maskX, vs->d_FX, nX);
    for (int g = 0; g < vs->ngroups && st == FE_OK; ++g)
      if (vs->group_lpc[g]) st = lpc_set_scaling(vs->group_lpc[g], vs->d_FX, s);
  }
  if (st == FE_OK) st = cuda_error(cudaStreamSynchronize(s), "fe_vspace_set_learned: scaling");
  cudaFree(mult);
  return st;
}

bool vspace_lpc_complete(const fe_vspace* vs, int op) {
  if (vs->lpc_op != op) return false;
  for (int g = 0; g < vs->ngroups; ++g)
    if (!vs->group_lpc[g]) return false;
  return true;
}

// z = M(r) on true dofs: r taken zero and z zeroed on the boundary (M = (1-m) M (1-m)).
int vspace_lpc_apply(fe_vspace* vs, const double* r, double* z, cudaStream_t s) {
  cudaError_t err0;
  if (!vs->d_rm && (err0 = cudaMalloc(&vs->d_rm, sizeof(double) * vs->ntrue)) != cudaSuccess) {
    vs->d_rm = nullptr;
    return cuda_error(err0, "fe_vspace: learned preconditioner workspace");
  }
  k_mask_copy<<<grid_of(vs->ntrue), 256, 0, s>>>(r, vs->d_mask, vs->d_rm, vs->ntrue);
  int st = fill_X(vs, vs->d_rm, s);
  if (st != FE_OK) return st;
  cudaError_t err = cudaMemsetAsync(vs->d_Y, 0, sizeof(double) * (vs->ntrue + vs->nc), s);
  if (err != cudaSuccess) return cuda_error(err, "fe_vspace: zero Y");
  for (int g = 0; g < vs->ngroups; ++g)
    if ((st = lpc_apply(vs->group_lpc[g], vs->d_X, vs->d_Y, s, true)) != FE_OK) return st;
  if ((st = fold_Y(vs, z, 0, s)) != FE_OK) return st;
  k_mask_zero<<<grid_of(vs->ntrue), 256, 0, s>>>(z, vs->d_mask, vs->ntrue);
  return cuda_error(cudaGetLastError(), "fe_vspace: learned preconditioner");
}

}  // namespace

extern "C" {

int fe_vspace_set_learned(fe_vspace* vs, int op, int order, const fe_lpc* trained, void* stream) {
  clear_error();
  if (!vs) return set_error(FE_ERR_ARG, "fe_vspace_set_learned: vs is NULL");
  if (op != FE_DIFFUSION && op != FE_MASS) return set_error(FE_ERR_ARG, "fe_vspace_set_learned: bad op");
  if (!(vs->ops & op))
    return set_error(FE_ERR_ARG, "fe_vspace_set_learned: operator not set up in fe_vspace_setup");
  int g = -1;
  for (int k = 0; k < vs->ngroups; ++k)
    if (vs->group_p[k] == order) g = k;
  if (g < 0) return set_error(FE_ERR_ARG, "fe_vspace_set_learned: no element of this order");
  cudaStream_t s = (cudaStream_t)stream;
  if (vs->lpc_op != op) {  // networks of another operator are dropped
    for (int k = 0; k < vs->ngroups; ++k) {
      fe_lpc_destroy(vs->group_lpc[k]);
      vs->group_lpc[k] = nullptr;
    }
    vs->lpc_op = op;
  }
  if (!trained) {
    fe_lpc_destroy(vs->group_lpc[g]);
    vs->group_lpc[g] = nullptr;
    return FE_OK;
  }
  int to = 0, tdin = 0, tw = 0;
  lpc_shape(trained, &to, &tdin, &tw);
  if (to != order) return set_error(FE_ERR_ARG, "fe_vspace_set_learned: network of another order");
  int cw = -1;
  if (vs->group_lpc[g]) lpc_shape(vs->group_lpc[g], nullptr, nullptr, &cw);
  if (cw != tw) {
    fe_lpc_destroy(vs->group_lpc[g]);
    vs->group_lpc[g] = nullptr;
    int st = fe_lpc_create(vs->group_pa[g], op, tw, 1, &vs->group_lpc[g]);
    if (st != FE_OK) {
      vs->group_lpc[g] = nullptr;
      return st;
    }
  }
  int st = lpc_copy_weights(vs->group_lpc[g], trained, s);
  if (st == FE_OK) st = vspace_lpc_scaling(vs, op, s);
  return st;
}

int fe_vspace_lpc_apply(fe_vspace* vs, const double* dev_r, double* dev_z, void* stream) {
  clear_error();
  if (!vs || !dev_r || !dev_z) return set_error(FE_ERR_ARG, "fe_vspace_lpc_apply: null argument");
  if (!vspace_lpc_complete(vs, vs->lpc_op))
    return set_error(FE_ERR_UNSUPPORTED, "fe_vspace_lpc_apply: a network is missing for an order");
  return vspace_lpc_apply(vs, dev_r, dev_z, (cudaStream_t)stream);
}

int fe_vspace_fcg(fe_vspace* vs, int op, const double* dev_b, double* dev_x, double rtol,
                  int maxit, fe_pcg_stats* stats, void* stream) {
  clear_error();
  if (stats) *stats = fe_pcg_stats{0, 0.0, 0.0, 0.0, 0, 0};
  if (!vs || !dev_b || !dev_x) return set_error(FE_ERR_ARG, "fe_vspace_fcg: null argument");
  if (op != FE_DIFFUSION && op != FE_MASS) return set_error(FE_ERR_ARG, "fe_vspace_fcg: bad op");
  if (!(vs->ops & op)) return set_error(FE_ERR_ARG, "fe_vspace_fcg: operator not set up");
  if (maxit < 1 || !(rtol >= 0.0)) return set_error(FE_ERR_ARG, "fe_vspace_fcg: bad rtol or maxit");
  if (!vspace_lpc_complete(vs, op))
    return set_error(FE_ERR_UNSUPPORTED, "fe_vspace_fcg: attach a network to every order first "
                                         "(fe_vspace_set_learned)");
  for (int g = 0; g < vs->ngroups; ++g)
    if (vs->group_pa[g]->variant == FE_VARIANT_F32)
      return set_error(FE_ERR_UNSUPPORTED, "fe_vspace_fcg: the FP32 variant is not FP64-accurate");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = vs->ntrue;
  double *dinv = nullptr, *diag = nullptr;
  int* flag = nullptr;
  cudaError_t err;
  if ((err = cudaMalloc(&dinv, sizeof(double) * n)) != cudaSuccess ||
      (err = cudaMalloc(&diag, sizeof(double) * n)) != cudaSuccess ||
      (err = cudaMalloc(&flag, sizeof(int))) != cudaSuccess) {
    cudaFree(dinv);
    cudaFree(diag);
    return cuda_error(err, "fe_vspace_fcg: cudaMalloc");
  }
  // the Jacobi fallback's inverse diagonal of E^T diag(A_E) E (0 on the boundary)
  int st = fe_vspace_diagonal(vs, op, diag, stream);
  if (st == FE_OK) {
    cudaMemsetAsync(flag, 0, sizeof(int), s);
    k_vs_dinv<<<grid_of(n), 256, 0, s>>>(diag, vs->d_mask, dinv, n, flag);
    st = cuda_error(cudaGetLastError(), "fe_vspace_fcg: diagonal");
  }
  if (st == FE_OK) {
    FcgOperator A;
    A.n = n;
    A.mask = vs->d_mask;
    A.apply = [&](const double* in, double* out) { return vspace_apply(vs, op, -1, in, out, s); };
    A.prec = [&](const double* r, double* z) { return vspace_lpc_apply(vs, r, z, s); };
    A.true_apply = [&](const double* in, double* out) {
      return vspace_apply(vs, op, FE_VARIANT_F64, in, out, s);
    };
    st = fcg_solve(A, dinv, dev_b, dev_x, rtol, maxit, s, stats, "fe_vspace_fcg");
  }
  cudaFree(dinv);
  cudaFree(diag);
  cudaFree(flag);
  return st;
}

}  // extern "C"
