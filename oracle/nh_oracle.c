/*
 * nh_oracle.c -- plain FP64 reference of the finite-strain solid element
 * loop: total Lagrangian, first Piola-Kirchhoff stress.  TEST INFRASTRUCTURE
 * ONLY: called by the tests and the smoke check, never by the engine, and it
 * shares no code with it.
 *
 * The paper's structure solver (Sec. 2.2) balances momentum in the reference
 * configuration, rho0 d2u/dt2 - Div P = b0, with P the first Piola-Kirchhoff
 * stress; Galerkin in space, Newmark in time and Newton-Raphson iterations,
 * each of which assembles the Jacobian A and the residual b.  The paper names
 * no material.  The reading here is the compressible neo-Hookean solid
 * (Bonet and Wood, "Nonlinear Continuum Mechanics for Finite Element
 * Analysis", 2nd ed., 2008, Sec. 6.4.3), written from its energy:
 *
 *     Psi(F) = mu/2 (F:F - 3) - mu ln J + lam/2 (ln J)^2,     J = det F > 0,
 *     P      = dPsi/dF   = mu (F - F^-T) + lam ln J F^-T,
 *     A_iJkL = dP_iJ/dF_kL
 *            = mu d_ik d_JL + lam F^-1_Ji F^-1_Lk + (mu - lam ln J) F^-1_Jk F^-1_Li.
 *
 * Per element, with grad0 N_a the reference gradients and, at each Gauss
 * point, F = I + sum_a u_a (x) grad0 N_a:
 *
 *     A^e_(a i),(b k) = sum_q w_q detJ0_q [ sum_{J,L} d_J N_a A_iJkL d_L N_b + m N_a N_b d_ik ],
 *     b^e_(a i)       = sum_q w_q detJ0_q sum_J P_iJ d_J N_a          (internal force),
 *
 * the mass term being the inertia part of the Newmark Jacobian,
 * m = rho0 / (beta dt^2) >= 0 (0: a static Newton step).  Material
 * parameters prm[]: E, nu, m.  The tet4 rule is always the 4-point one.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

int oracle_quadrature(int type, int tet_rule, double* pts, double* w);
int oracle_shape(int type, const double* p, double* N, double* dN);

#define NH_MAXN 8
#define NH_MAXQ 8

static int nh_nodes(int type) { return type == 0 ? 4 : type == 1 ? 5 : type == 2 ? 6 : 8; }

static void nh_lame(const double* prm, double* lam, double* mu) {
  const double E = prm[0], nu = prm[1];
  *lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  *mu = E / (2.0 * (1.0 + nu));
}

/* inverse of a 3x3 matrix (row-major) and its determinant */
static double inv3(const double* M, double* Mi) {
  const double c00 = M[4] * M[8] - M[5] * M[7];
  const double c01 = M[5] * M[6] - M[3] * M[8];
  const double c02 = M[3] * M[7] - M[4] * M[6];
  const double det = M[0] * c00 + M[1] * c01 + M[2] * c02;
  Mi[0] = c00 / det;
  Mi[1] = (M[2] * M[7] - M[1] * M[8]) / det;
  Mi[2] = (M[1] * M[5] - M[2] * M[4]) / det;
  Mi[3] = c01 / det;
  Mi[4] = (M[0] * M[8] - M[2] * M[6]) / det;
  Mi[5] = (M[2] * M[3] - M[0] * M[5]) / det;
  Mi[6] = c02 / det;
  Mi[7] = (M[1] * M[6] - M[0] * M[7]) / det;
  Mi[8] = (M[0] * M[4] - M[1] * M[3]) / det;
  return det;
}

/* ---------------------------------------------------------------------------
 * The material at one point.  F: 3x3 row-major (F_iJ at 3 i + J).  Writes P
 * (3x3), the tangent Aten[((i*3 + J)*3 + k)*3 + L] (may be NULL) and the
 * energy density *psi (may be NULL).  Returns 0, or 1 when det F <= 0.
 * ------------------------------------------------------------------------- */
int oracle_nh_point(const double* prm, const double* F, double* P, double* Aten, double* psi) {
  double lam, mu;
  nh_lame(prm, &lam, &mu);
  double Fi[9];
  const double J = inv3(F, Fi);
  if (!(J > 0.0)) return 1;
  const double lnJ = log(J);
  /* F^-T_iJ = F^-1_Ji */
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) P[3 * i + j] = mu * (F[3 * i + j] - Fi[3 * j + i]) + lam * lnJ * Fi[3 * j + i];
  if (Aten)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k)
          for (int l = 0; l < 3; ++l)
            Aten[((i * 3 + j) * 3 + k) * 3 + l] = (i == k && j == l ? mu : 0.0) + lam * Fi[3 * j + i] * Fi[3 * l + k] +
                                                  (mu - lam * lnJ) * Fi[3 * j + k] * Fi[3 * l + i];
  if (psi) {
    double ff = 0.0;
    for (int t = 0; t < 9; ++t) ff += F[t] * F[t];
    *psi = 0.5 * mu * (ff - 3.0) - mu * lnJ + 0.5 * lam * lnJ * lnJ;
  }
  return 0;
}

/* ---------------------------------------------------------------------------
 * Element Jacobian, internal force and stored energy.  X, U: [nn][3] reference
 * coordinates and displacements.  Ne / Nb (may be NULL): normwise error
 * scales |w detJ0| (mu |g_a||g_b| + (|lam| + |mu - lam ln J|) |h_a||h_b| +
 * |m| |N_a N_b|) and |w detJ0| |P|_F |g_a|, with g_a = grad0 N_a and
 * h_a = F^-T g_a.  energy (may be NULL): sum_q w detJ0 Psi.
 * Returns 0, 1 for det J0 <= 0, 3 for det F <= 0.
 * ------------------------------------------------------------------------- */
int oracle_nh_element(int type, const double* prm, const double* X, const double* U, double* Ae, double* be,
                      double* Ne, double* Nb, double* energy) {
  const int nn = nh_nodes(type), n = 3 * nn;
  double pts[NH_MAXQ * 3], w[NH_MAXQ];
  const int nq = oracle_quadrature(type, 1, pts, w);
  double lam, mu;
  nh_lame(prm, &lam, &mu);
  const double m = prm[2];
  memset(Ae, 0, sizeof(double) * n * n);
  memset(be, 0, sizeof(double) * n);
  if (Ne) memset(Ne, 0, sizeof(double) * n * n);
  if (Nb) memset(Nb, 0, sizeof(double) * n);
  if (energy) *energy = 0.0;
  for (int q = 0; q < nq; ++q) {
    double N[NH_MAXN], dN[NH_MAXN * 3];
    oracle_shape(type, pts + 3 * q, N, dN);
    double J0[9] = {0};
    for (int a = 0; a < nn; ++a)
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) J0[3 * i + j] += X[3 * a + i] * dN[3 * a + j];
    double J0i[9];
    const double det0 = inv3(J0, J0i);
    if (!(det0 > 0.0)) return 1;
    /* reference gradients g_a = J0^-T grad_xi N_a */
    double g[NH_MAXN][3];
    for (int a = 0; a < nn; ++a)
      for (int i = 0; i < 3; ++i) {
        g[a][i] = 0.0;
        for (int j = 0; j < 3; ++j) g[a][i] += J0i[3 * j + i] * dN[3 * a + j];
      }
    double F[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    for (int a = 0; a < nn; ++a)
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) F[3 * i + j] += U[3 * a + i] * g[a][j];
    double P[9], At[81], psi;
    if (oracle_nh_point(prm, F, P, At, &psi)) return 3;
    const double wd = w[q] * det0;
    if (energy) *energy += wd * psi;
    for (int a = 0; a < nn; ++a)
      for (int b = 0; b < nn; ++b)
        for (int i = 0; i < 3; ++i)
          for (int k = 0; k < 3; ++k) {
            double s = 0.0;
            for (int j = 0; j < 3; ++j)
              for (int l = 0; l < 3; ++l) s += g[a][j] * At[((i * 3 + j) * 3 + k) * 3 + l] * g[b][l];
            if (i == k) s += m * N[a] * N[b];
            Ae[(3 * a + i) * n + 3 * b + k] += wd * s;
          }
    for (int a = 0; a < nn; ++a)
      for (int i = 0; i < 3; ++i) {
        double s = 0.0;
        for (int j = 0; j < 3; ++j) s += P[3 * i + j] * g[a][j];
        be[3 * a + i] += wd * s;
      }
    if (Ne || Nb) {
      double Fi[9];
      const double J = inv3(F, Fi);
      const double lnJ = log(J);
      double gn[NH_MAXN], hn[NH_MAXN];
      for (int a = 0; a < nn; ++a) {
        double h2 = 0.0, g2 = 0.0;
        for (int i = 0; i < 3; ++i) {
          double h = 0.0;
          for (int j = 0; j < 3; ++j) h += Fi[3 * j + i] * g[a][j];
          h2 += h * h;
          g2 += g[a][i] * g[a][i];
        }
        gn[a] = sqrt(g2);
        hn[a] = sqrt(h2);
      }
      double pn = 0.0;
      for (int t = 0; t < 9; ++t) pn += P[t] * P[t];
      pn = sqrt(pn);
      const double cl = fabs(lam) + fabs(mu - lam * lnJ);
      for (int a = 0; a < nn; ++a) {
        if (Nb)
          for (int i = 0; i < 3; ++i) Nb[3 * a + i] += fabs(wd) * pn * gn[a];
        if (Ne)
          for (int b = 0; b < nn; ++b) {
            const double s = fabs(wd) * (mu * gn[a] * gn[b] + cl * hn[a] * hn[b] + fabs(m) * fabs(N[a] * N[b]));
            for (int i = 0; i < 3; ++i)
              for (int k = 0; k < 3; ++k) Ne[(3 * a + i) * n + 3 * b + k] += s;
          }
      }
    }
  }
  return 0;
}

/* ---------------------------------------------------------------------------
 * Jacobian + internal force of the whole mesh in element-index order, over
 * the oracle's own pattern (rp_s: scalar row_ptr, node_map: rank map), 3 dofs
 * per node.  U: [n_nodes][3].  energy (may be NULL): the stored energy.
 * Returns 0, -(e+1) when element e is inverted in the reference
 * configuration, -(E+e+1) when its deformation is (det F <= 0).
 * ------------------------------------------------------------------------- */
int64_t oracle_nh_assemble(int64_t n_nodes, int64_t n_elems, const uint8_t* types, const int64_t* conn_off,
                           const int32_t* conn, const double* coords, const double* prm, const double* U,
                           const int64_t* rp_s, const int32_t* node_map, double* A, double* b, double* NA, double* Nb,
                           double* energy) {
  (void)n_nodes;
  double X[3 * NH_MAXN], Ue[3 * NH_MAXN];
  double Ae[24 * 24], be[24], Ne[24 * 24], Nbe[24], en;
  int64_t off = 0;
  if (energy) *energy = 0.0;
  for (int64_t e = 0; e < n_elems; ++e) {
    const int ne = (int)(conn_off[e + 1] - conn_off[e]);
    const int32_t* cn = conn + conn_off[e];
    for (int a = 0; a < ne; ++a)
      for (int i = 0; i < 3; ++i) {
        X[3 * a + i] = coords[3 * (int64_t)cn[a] + i];
        Ue[3 * a + i] = U[3 * (int64_t)cn[a] + i];
      }
    const int rc = oracle_nh_element(types[e], prm, X, Ue, Ae, be, NA ? Ne : NULL, Nb ? Nbe : NULL, &en);
    if (rc == 1) return -(e + 1);
    if (rc == 3) return -(n_elems + e + 1);
    if (energy) *energy += en;
    const int n = 3 * ne;
    for (int a = 0; a < ne; ++a)
      for (int c = 0; c < 3; ++c) {
        const int64_t row = 3 * (int64_t)cn[a] + c;
        for (int bb = 0; bb < ne; ++bb) {
          const int64_t k = node_map[off + a * ne + bb];
          for (int cc = 0; cc < 3; ++cc) {
            const int64_t pos = rp_s[row] + 3 * k + cc;
            A[pos] += Ae[(3 * a + c) * n + 3 * bb + cc];
            if (NA) NA[pos] += Ne[(3 * a + c) * n + 3 * bb + cc];
          }
        }
        b[row] += be[3 * a + c];
        if (Nb) Nb[row] += Nbe[3 * a + c];
      }
    off += (int64_t)ne * ne;
  }
  return 0;
}
