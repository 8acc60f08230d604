/*
 * Sum-factorised partial-assembly operators on the CPU, FP64, OpenMP over elements
 * (oracle; TEST INFRASTRUCTURE -- the timed CPU baseline, never part of the library).
 *
 * The same operator as oracle/element.py + oracle/operator.py (the Galerkin definition), reached
 * the way the paper's Section II-B describes: the operator D at the quadrature points is stored
 * once ("partial assembly"), and the tensor-product basis of Eq. (2) is applied on the fly as
 * 1D contractions, one direction at a time, forward (B, G) and transposed (B^T, G^T) around the
 * pointwise D; the element restriction G of Eq. (1) is the gather through the dof numbering and
 * its transpose the scatter-add.  Standard forms for the H1 operators (the paper is silent on
 * them):
 *   diffusion  D_q = w_q c_e adj(J) adj(J)^T / det J   (symmetric, 6 entries per point)
 *   mass       M_q = w_q c_e det J
 * Everything here is written from those definitions: no blocking, fusion or reordering beyond
 * the sum factorisation itself.  Elements are processed in eight colours (parity of the element
 * coordinates); elements of one colour share no dof, so the scatter-add needs no atomics and the
 * result does not depend on the thread count.
 *
 * Numbering (as oracle/mesh.py): elements e = ex + nx (ey + ny ez); local dofs
 * a = i + D (j + D k); global dofs (ex p + i) + Nx ((ey p + j) + Ny (ez p + k)); vertices on the
 * (nx+1)(ny+1)(nz+1) lattice, x fastest; corner v = a + 2b + 4c at lattice offset (a, b, c).
 * Tables: B[q*D + d] = l_d(x_q), G[q*D + d] = l_d'(x_q) (from oracle/quadrature.py), Gauss
 * points pts[q] and weights wts[q] on [0, 1].
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define MAXD 9
#define MAXQ 10

int sf_threads(void) { return omp_get_max_threads(); }

/* Trilinear map of element (ex, ey, ez) at reference point (s, t, u): Jacobian
 * J[i][r] = d x_i / d xi_r. */
static void jacobian(const double* V, int nx, int ny, int ex, int ey, int ez, double s, double t,
                     double u, double J[3][3]) {
  memset(J, 0, 9 * sizeof(double));
  for (int v = 0; v < 8; ++v) {
    const int a = v & 1, b = (v >> 1) & 1, c = v >> 2;
    const int64_t idx = (ex + a) + (int64_t)(nx + 1) * ((ey + b) + (int64_t)(ny + 1) * (ez + c));
    const double fa = a ? s : 1.0 - s, fb = b ? t : 1.0 - t, fc = c ? u : 1.0 - u;
    const double da = a ? 1.0 : -1.0, db = b ? 1.0 : -1.0, dc = c ? 1.0 : -1.0;
    const double dN[3] = {da * fb * fc, fa * db * fc, fa * fb * dc};
    for (int i = 0; i < 3; ++i)
      for (int r = 0; r < 3; ++r) J[i][r] += V[3 * idx + i] * dN[r];
  }
}

/* Quadrature data of every element.  kind 1 (diffusion): out[e][q][6] = D_q entries
 * (xx, xy, xz, yy, yz, zz); kind 2 (mass): out[e][q] = M_q; q = qx + Q (qy + Q qz).  coeff: [ne]
 * or NULL for 1.  Returns the number of points with det J <= 0 (0 when the mesh is valid). */
int64_t sf_qdata(int nx, int ny, int nz, int Q, const double* pts, const double* wts,
                 const double* V, const double* coeff, int kind, double* out) {
  const int64_t ne = (int64_t)nx * ny * nz;
  const int Q3 = Q * Q * Q;
  int64_t bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
  for (int64_t e = 0; e < ne; ++e) {
    const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((int64_t)nx * ny));
    const double c = coeff ? coeff[e] : 1.0;
    for (int q = 0; q < Q3; ++q) {
      const int qx = q % Q, qy = (q / Q) % Q, qz = q / (Q * Q);
      double J[3][3];
      jacobian(V, nx, ny, ex, ey, ez, pts[qx], pts[qy], pts[qz], J);
      /* adj(J) = det(J) J^{-1}: adj[r][i] is the cofactor of J[i][r] */
      double adj[3][3];
      adj[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
      adj[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
      adj[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
      adj[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
      adj[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
      adj[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
      adj[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
      adj[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
      adj[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
      const double det = J[0][0] * adj[0][0] + J[0][1] * adj[1][0] + J[0][2] * adj[2][0];
      if (!(det > 0.0)) ++bad;
      const double w = wts[qx] * wts[qy] * wts[qz] * c;
      if (kind == 2) {
        out[e * Q3 + q] = w * det;
      } else {
        double* d = out + (e * Q3 + q) * 6;
        const int rr[6] = {0, 0, 0, 1, 1, 2}, ss[6] = {0, 1, 2, 1, 2, 2};
        for (int m = 0; m < 6; ++m) {
          double acc = 0.0;
          for (int i = 0; i < 3; ++i) acc += adj[rr[m]][i] * adj[ss[m]][i];
          d[m] = w * acc / det;
        }
      }
    }
  }
  return bad;
}

static int64_t gdof(int nx, int ny, int p, int ex, int ey, int ez, int i, int j, int k) {
  const int64_t Nx = (int64_t)nx * p + 1, Ny = (int64_t)ny * p + 1;
  return (ex * (int64_t)p + i) + Nx * ((ey * (int64_t)p + j) + Ny * (ez * (int64_t)p + k));
}

/* y_e = A_e x_e for one element by sum factorisation (ye, xe: [k][j][i]). */
static void elem_apply(int D, int Q, const double* B, const double* G, const double* qd,
                       int kind, const double* xe, double* ye) {
  double Tb[MAXD][MAXD][MAXQ], Tg[MAXD][MAXD][MAXQ];    /* [k][j][qx] */
  double Y0[MAXD][MAXQ][MAXQ], Y1[MAXD][MAXQ][MAXQ], Y2[MAXD][MAXQ][MAXQ]; /* [k][qy][qx] */
  double U0[MAXQ][MAXQ][MAXQ], U1[MAXQ][MAXQ][MAXQ], U2[MAXQ][MAXQ][MAXQ]; /* [qz][qy][qx] */
  /* x direction: Tb = B x, Tg = G x */
  for (int k = 0; k < D; ++k)
    for (int j = 0; j < D; ++j)
      for (int qx = 0; qx < Q; ++qx) {
        double sb = 0.0, sg = 0.0;
        for (int i = 0; i < D; ++i) {
          const double v = xe[(k * D + j) * D + i];
          sb += B[qx * D + i] * v;
          sg += G[qx * D + i] * v;
        }
        Tb[k][j][qx] = sb;
        Tg[k][j][qx] = sg;
      }
  if (kind == 2) {
    /* mass: U = (B x B x B) x, V = M U, y = (B x B x B)^T V */
    for (int k = 0; k < D; ++k)
      for (int qy = 0; qy < Q; ++qy)
        for (int qx = 0; qx < Q; ++qx) {
          double s = 0.0;
          for (int j = 0; j < D; ++j) s += B[qy * D + j] * Tb[k][j][qx];
          Y0[k][qy][qx] = s;
        }
    for (int qz = 0; qz < Q; ++qz)
      for (int qy = 0; qy < Q; ++qy)
        for (int qx = 0; qx < Q; ++qx) {
          double s = 0.0;
          for (int k = 0; k < D; ++k) s += B[qz * D + k] * Y0[k][qy][qx];
          U0[qz][qy][qx] = s * qd[(qz * Q + qy) * Q + qx];
        }
    for (int k = 0; k < D; ++k)
      for (int qy = 0; qy < Q; ++qy)
        for (int qx = 0; qx < Q; ++qx) {
          double s = 0.0;
          for (int qz = 0; qz < Q; ++qz) s += B[qz * D + k] * U0[qz][qy][qx];
          Y0[k][qy][qx] = s;
        }
    for (int k = 0; k < D; ++k)
      for (int j = 0; j < D; ++j)
        for (int qx = 0; qx < Q; ++qx) {
          double s = 0.0;
          for (int qy = 0; qy < Q; ++qy) s += B[qy * D + j] * Y0[k][qy][qx];
          Tb[k][j][qx] = s;
        }
    for (int k = 0; k < D; ++k)
      for (int j = 0; j < D; ++j)
        for (int i = 0; i < D; ++i) {
          double s = 0.0;
          for (int qx = 0; qx < Q; ++qx) s += B[qx * D + i] * Tb[k][j][qx];
          ye[(k * D + j) * D + i] = s;
        }
    return;
  }
  /* diffusion: reference gradient u_r = d/dxi_r at the points (G along axis r, B elsewhere) */
  for (int k = 0; k < D; ++k)
    for (int qy = 0; qy < Q; ++qy)
      for (int qx = 0; qx < Q; ++qx) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        for (int j = 0; j < D; ++j) {
          s0 += B[qy * D + j] * Tg[k][j][qx];
          s1 += G[qy * D + j] * Tb[k][j][qx];
          s2 += B[qy * D + j] * Tb[k][j][qx];
        }
        Y0[k][qy][qx] = s0;
        Y1[k][qy][qx] = s1;
        Y2[k][qy][qx] = s2;
      }
  for (int qz = 0; qz < Q; ++qz)
    for (int qy = 0; qy < Q; ++qy)
      for (int qx = 0; qx < Q; ++qx) {
        double u0 = 0.0, u1 = 0.0, u2 = 0.0;
        for (int k = 0; k < D; ++k) {
          u0 += B[qz * D + k] * Y0[k][qy][qx];
          u1 += B[qz * D + k] * Y1[k][qy][qx];
          u2 += G[qz * D + k] * Y2[k][qy][qx];
        }
        /* v = D_q u, D_q symmetric (xx, xy, xz, yy, yz, zz) */
        const double* d = qd + ((qz * Q + qy) * Q + qx) * 6;
        U0[qz][qy][qx] = d[0] * u0 + d[1] * u1 + d[2] * u2;
        U1[qz][qy][qx] = d[1] * u0 + d[3] * u1 + d[4] * u2;
        U2[qz][qy][qx] = d[2] * u0 + d[4] * u1 + d[5] * u2;
      }
  /* transposed: y = sum_r (d/dxi_r)^T v_r */
  for (int k = 0; k < D; ++k)
    for (int qy = 0; qy < Q; ++qy)
      for (int qx = 0; qx < Q; ++qx) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        for (int qz = 0; qz < Q; ++qz) {
          s0 += B[qz * D + k] * U0[qz][qy][qx];
          s1 += B[qz * D + k] * U1[qz][qy][qx];
          s2 += G[qz * D + k] * U2[qz][qy][qx];
        }
        Y0[k][qy][qx] = s0;
        Y1[k][qy][qx] = s1;
        Y2[k][qy][qx] = s2;
      }
  for (int k = 0; k < D; ++k)
    for (int j = 0; j < D; ++j)
      for (int qx = 0; qx < Q; ++qx) {
        double s0 = 0.0, s12 = 0.0;
        for (int qy = 0; qy < Q; ++qy) {
          s0 += B[qy * D + j] * Y0[k][qy][qx];
          s12 += G[qy * D + j] * Y1[k][qy][qx] + B[qy * D + j] * Y2[k][qy][qx];
        }
        Tg[k][j][qx] = s0;   /* to be contracted with G^T along x */
        Tb[k][j][qx] = s12;  /* to be contracted with B^T along x */
      }
  for (int k = 0; k < D; ++k)
    for (int j = 0; j < D; ++j)
      for (int i = 0; i < D; ++i) {
        double s = 0.0;
        for (int qx = 0; qx < Q; ++qx) s += G[qx * D + i] * Tg[k][j][qx] + B[qx * D + i] * Tb[k][j][qx];
        ye[(k * D + j) * D + i] = s;
      }
}

/* y = A x (full L-vector, no boundary conditions): y zeroed, then every element's A_e x_e
 * scatter-added, colour by colour.  kind 1 diffusion, 2 mass; qd as sf_qdata wrote it. */
void sf_apply(int nx, int ny, int nz, int p, int Q, const double* B, const double* G,
              const double* qd, int kind, const double* x, double* y) {
  const int D = p + 1;
  const int64_t nd = ((int64_t)nx * p + 1) * ((int64_t)ny * p + 1) * ((int64_t)nz * p + 1);
  const int per = (kind == 2 ? 1 : 6) * Q * Q * Q;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < nd; ++i) y[i] = 0.0;
  for (int colour = 0; colour < 8; ++colour) {
    const int cx = colour & 1, cy = (colour >> 1) & 1, cz = colour >> 2;
    const int mx = (nx - cx + 1) / 2, my = (ny - cy + 1) / 2, mz = (nz - cz + 1) / 2;
    const int64_t m = (int64_t)mx * my * mz;
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < m; ++t) {
      const int ex = cx + 2 * (int)(t % mx), ey = cy + 2 * (int)((t / mx) % my);
      const int ez = cz + 2 * (int)(t / ((int64_t)mx * my));
      const int64_t e = ex + (int64_t)nx * (ey + (int64_t)ny * ez);
      double xe[MAXD * MAXD * MAXD], ye[MAXD * MAXD * MAXD];
      for (int k = 0; k < D; ++k)
        for (int j = 0; j < D; ++j)
          for (int i = 0; i < D; ++i)
            xe[(k * D + j) * D + i] = x[gdof(nx, ny, p, ex, ey, ez, i, j, k)];
      elem_apply(D, Q, B, G, qd + e * per, kind, xe, ye);
      for (int k = 0; k < D; ++k)
        for (int j = 0; j < D; ++j)
          for (int i = 0; i < D; ++i) y[gdof(nx, ny, p, ex, ey, ez, i, j, k)] += ye[(k * D + j) * D + i];
    }
  }
}

/* diag(A) from the definition: diag_e[a] = sum_q sum_rs D_q^{rs} dphi_a/dxi_r dphi_a/dxi_s (or
 * M_q phi_a^2), scatter-added colour by colour. */
void sf_diagonal(int nx, int ny, int nz, int p, int Q, const double* B, const double* G,
                 const double* qd, int kind, double* diag) {
  const int D = p + 1;
  const int64_t nd = ((int64_t)nx * p + 1) * ((int64_t)ny * p + 1) * ((int64_t)nz * p + 1);
  const int per = (kind == 2 ? 1 : 6) * Q * Q * Q;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < nd; ++i) diag[i] = 0.0;
  for (int colour = 0; colour < 8; ++colour) {
    const int cx = colour & 1, cy = (colour >> 1) & 1, cz = colour >> 2;
    const int mx = (nx - cx + 1) / 2, my = (ny - cy + 1) / 2, mz = (nz - cz + 1) / 2;
    const int64_t m = (int64_t)mx * my * mz;
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < m; ++t) {
      const int ex = cx + 2 * (int)(t % mx), ey = cy + 2 * (int)((t / mx) % my);
      const int ez = cz + 2 * (int)(t / ((int64_t)mx * my));
      const int64_t e = ex + (int64_t)nx * (ey + (int64_t)ny * ez);
      const double* q0 = qd + e * per;
      for (int k = 0; k < D; ++k)
        for (int j = 0; j < D; ++j)
          for (int i = 0; i < D; ++i) {
            double s = 0.0;
            for (int qz = 0; qz < Q; ++qz)
              for (int qy = 0; qy < Q; ++qy)
                for (int qx = 0; qx < Q; ++qx) {
                  const int q = (qz * Q + qy) * Q + qx;
                  const double bx = B[qx * D + i], by = B[qy * D + j], bz = B[qz * D + k];
                  if (kind == 2) {
                    const double ph = bx * by * bz;
                    s += q0[q] * ph * ph;
                  } else {
                    const double g[3] = {G[qx * D + i] * by * bz, bx * G[qy * D + j] * bz,
                                         bx * by * G[qz * D + k]};
                    const double* d = q0 + q * 6;
                    s += d[0] * g[0] * g[0] + d[3] * g[1] * g[1] + d[5] * g[2] * g[2] +
                         2.0 * (d[1] * g[0] * g[1] + d[2] * g[0] * g[2] + d[4] * g[1] * g[2]);
                  }
                }
            diag[gdof(nx, ny, p, ex, ey, ez, i, j, k)] += s;
          }
    }
  }
}

/* Jacobi-preconditioned CG for A_bc x = b, A_bc = (1-m) A (1-m) + m, from x = 0, b's boundary
 * entries ignored; stops when ||r||_2 <= rtol ||(1-m) b||_2 or after maxit iterations.  work:
 * 4 vectors of ndofs (r, z, p, q).  FP64 throughout; the inner products are OpenMP reductions.
 * Returns the iterations; *rel = the final ||r|| / ||(1-m) b||. */
int sf_pcg(int nx, int ny, int nz, int p, int Q, const double* B, const double* G,
           const double* qd, int kind, const unsigned char* mask, const double* diag,
           const double* b, double* x, double rtol, int maxit, double* work, double* rel) {
  const int64_t nd = ((int64_t)nx * p + 1) * ((int64_t)ny * p + 1) * ((int64_t)nz * p + 1);
  double *r = work, *z = work + nd, *pv = work + 2 * nd, *q = work + 3 * nd;
  double rz = 0.0, bb = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : rz, bb)
  for (int64_t i = 0; i < nd; ++i) {
    const double bi = mask[i] ? 0.0 : b[i];
    x[i] = 0.0;
    r[i] = bi;
    z[i] = mask[i] ? 0.0 : bi / diag[i];
    pv[i] = z[i];
    rz += r[i] * z[i];
    bb += bi * bi;
  }
  *rel = bb > 0.0 ? 1.0 : 0.0;
  if (!(bb > 0.0)) return 0;
  int it = 0;
  while (it < maxit) {
    sf_apply(nx, ny, nz, p, Q, B, G, qd, kind, pv, q);
    double pq = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : pq)
    for (int64_t i = 0; i < nd; ++i) {
      if (mask[i]) q[i] = 0.0;
      pq += pv[i] * q[i];
    }
    if (!(pq > 0.0)) break;
    const double alpha = rz / pq;
    double rz1 = 0.0, rr = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : rz1, rr)
    for (int64_t i = 0; i < nd; ++i) {
      x[i] += alpha * pv[i];
      r[i] -= alpha * q[i];
      z[i] = mask[i] ? 0.0 : r[i] / diag[i];
      rz1 += r[i] * z[i];
      rr += r[i] * r[i];
    }
    ++it;
    *rel = sqrt(rr / bb);
    if (*rel <= rtol) break;
    const double beta = rz1 / rz;
    rz = rz1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nd; ++i) pv[i] = z[i] + beta * pv[i];
  }
  return it;
}
