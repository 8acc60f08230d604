// 1D tables of the tensor-product basis (host side of libfe).
//
// Eq. (2) builds the 3D basis from one 1D matrix, B_abc,ijk = B1d_ai B1d_bj B1d_ck.  The nodes
// and rule are not fixed by the paper; libfe uses the standard H1 spectral-element choices:
// Lagrange polynomials on the p+1 Gauss-Lobatto-Legendre nodes of [0,1], evaluated at the
// q-point Gauss-Legendre rule.  Everything is computed in long double and rounded once.
#include <cmath>

#include "fe_internal.h"

namespace fe {
namespace {

typedef long double ld;

// Legendre P_n(x) and P_{n-1}(x) by the three-term recurrence.
void legendre_pair(int n, ld x, ld* pn, ld* pnm1) {
  ld a = 1.0L, b = x;  // P_0, P_1
  if (n == 0) { *pn = 1.0L; *pnm1 = 0.0L; return; }
  for (int k = 1; k < n; ++k) {
    ld c = ((2 * k + 1) * x * b - k * a) / (k + 1);
    a = b;
    b = c;
  }
  *pn = b;
  *pnm1 = a;
}

// Roots of P_n on (-1, 1), ascending, with Gauss weights 2 / ((1 - x^2) P_n'(x)^2).
void gauss_legendre_pm1(int n, ld* x, ld* w) {
  const ld pi = 3.141592653589793238462643383279502884L;
  for (int i = 0; i < n; ++i) {
    ld t = std::cos(pi * (i + 0.75L) / (n + 0.5L));
    for (int it = 0; it < 100; ++it) {
      ld pn, pm;
      legendre_pair(n, t, &pn, &pm);
      ld dp = n * (t * pn - pm) / (t * t - 1.0L);
      ld dt = pn / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-19L) break;
    }
    ld pn, pm;
    legendre_pair(n, t, &pn, &pm);
    ld dp = n * (t * pn - pm) / (t * t - 1.0L);
    x[n - 1 - i] = t;  // cos guesses are descending
    w[n - 1 - i] = 2.0L / ((1.0L - t * t) * dp * dp);
  }
}

// Gauss-Lobatto-Legendre nodes on [-1, 1] (d of them): +-1 and the roots of P_{d-1}'.
// Newton on f = (1 - x^2) P_n'(x) = n (P_{n-1} - x P_n), f' = -n (n + 1) P_n.
void gauss_lobatto_pm1(int d, ld* x) {
  const ld pi = 3.141592653589793238462643383279502884L;
  const int n = d - 1;
  x[0] = -1.0L;
  x[n] = 1.0L;
  for (int i = 1; i < n; ++i) {
    ld t = -std::cos(pi * i / n);
    for (int it = 0; it < 100; ++it) {
      ld pn, pm;
      legendre_pair(n, t, &pn, &pm);
      ld f = n * (pm - t * pn);
      ld df = -(ld)n * (n + 1) * pn;
      ld dt = f / df;
      t -= dt;
      if (std::fabs(dt) < 1e-19L) break;
    }
    x[i] = t;
  }
}

}  // namespace

bool make_basis_1d(int p, int q, Basis1D* out) {
  if (p < 1 || p > kMaxOrder || q < 1 || q > kMaxQ) return false;
  const int D = p + 1;
  ld nodes[kMaxD], gx[kMaxQ], gw[kMaxQ];
  gauss_lobatto_pm1(D, nodes);
  gauss_legendre_pm1(q, gx, gw);
  for (int d = 0; d < D; ++d) nodes[d] = (nodes[d] + 1.0L) / 2.0L;
  for (int i = 0; i < q; ++i) {
    gx[i] = (gx[i] + 1.0L) / 2.0L;
    gw[i] = gw[i] / 2.0L;
  }
  // barycentric weights lambda_d = 1 / prod_{m != d} (t_d - t_m)
  ld lam[kMaxD];
  for (int d = 0; d < D; ++d) {
    ld prod = 1.0L;
    for (int m = 0; m < D; ++m)
      if (m != d) prod *= nodes[d] - nodes[m];
    lam[d] = 1.0L / prod;
  }
  out->p = p;
  out->D = D;
  out->Q = q;
  for (int d = 0; d < D; ++d) out->nodes[d] = (double)nodes[d];
  for (int i = 0; i < q; ++i) {
    out->pts[i] = (double)gx[i];
    out->wts[i] = (double)gw[i];
    const ld x = gx[i];
    // l_d(x) = lambda_d * prod_{m != d} (x - t_m)  (first form of the barycentric formula),
    // l_d'(x) = l_d(x) * sum_{m != d} 1 / (x - t_m), evaluated without dividing by a vanishing
    // factor: sum over m of lambda_d * prod_{l != d, m} (x - t_l).
    for (int d = 0; d < D; ++d) {
      ld val = lam[d], der = 0.0L;
      for (int m = 0; m < D; ++m)
        if (m != d) val *= x - nodes[m];
      for (int m = 0; m < D; ++m) {
        if (m == d) continue;
        ld term = lam[d];
        for (int l = 0; l < D; ++l)
          if (l != d && l != m) term *= x - nodes[l];
        der += term;
      }
      out->B[i * D + d] = (double)val;
      out->G[i * D + d] = (double)der;
    }
  }
  return true;
}

bool make_l2_basis_1d(int p, int q, double* Bl) {
  if (p < 0 || p + 1 > kMaxD || q < 1 || q > kMaxQ) return false;
  const int D = p + 1;
  ld nodes[kMaxD], nw[kMaxD], gx[kMaxQ], gw[kMaxQ];
  gauss_legendre_pm1(D, nodes, nw);
  gauss_legendre_pm1(q, gx, gw);
  for (int d = 0; d < D; ++d) nodes[d] = (nodes[d] + 1.0L) / 2.0L;
  for (int i = 0; i < q; ++i) {
    const ld x = (gx[i] + 1.0L) / 2.0L;
    for (int d = 0; d < D; ++d) {
      ld val = 1.0L;
      for (int m = 0; m < D; ++m)
        if (m != d) val *= (x - nodes[m]) / (nodes[d] - nodes[m]);
      Bl[i * D + d] = (double)val;
    }
  }
  return true;
}

}  // namespace fe

extern "C" int fe_basis_1d(int order, int q1d, double* nodes, double* pts, double* wts,
                           double* B, double* G) {
  fe::clear_error();
  fe::Basis1D b;
  if (!fe::make_basis_1d(order, q1d, &b))
    return fe::set_error(FE_ERR_ARG, "fe_basis_1d: order must be 1..8 and q1d 1..10");
  const int D = b.D, Q = b.Q;
  for (int d = 0; d < D; ++d)
    if (nodes) nodes[d] = b.nodes[d];
  for (int i = 0; i < Q; ++i) {
    if (pts) pts[i] = b.pts[i];
    if (wts) wts[i] = b.wts[i];
    for (int d = 0; d < D; ++d) {
      if (B) B[i * D + d] = b.B[i * D + d];
      if (G) G[i * D + d] = b.G[i * D + d];
    }
  }
  return FE_OK;
}
