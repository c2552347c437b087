/*
 * j2_oracle.c -- plain FP64 reference of the elastoplastic (J2, Voce
 * hardening) element loop.  TEST INFRASTRUCTURE ONLY: called by the tests,
 * the smoke check and the fixture script under tests/golden, never by the
 * engine, and it shares no code with it.
 *
 * The paper's solid mechanics problem (Sec. 2.2) assembles, at every Newton
 * step of a nonlinear solid, the tangent matrix and the internal force
 * vector; the constitutive update at every Gauss point is the costly part of
 * that element loop (Sec. 5.2).  The paper names no material model; this is
 * the small-strain reading: J2 plasticity with isotropic Voce hardening
 *
 *     sigma_y(alpha) = sigma0 + H alpha + (sigma_inf - sigma0)(1 - exp(-delta alpha)),
 *
 * integrated by the radial-return map with its consistent tangent (Simo and
 * Hughes, "Computational Inelasticity", 1998, ch. 3; written here from the
 * derivation, see oracle_j2_point).  Per element:
 *
 *     A^e = sum_q w_q detJ_q B^T D_ep B,     b^e = f_int = sum_q w_q detJ_q B^T sigma
 *
 * with the strain eps = sym(grad u) of the nodal displacements u, Voigt order
 * (xx, yy, zz, xy, yz, xz) and engineering shear in B and D_ep.
 *
 * Gauss-point state, 7 values per point: the plastic strain tensor
 * components (xx, yy, zz, xy, yz, xz) and the equivalent plastic strain alpha.
 *
 * Material parameters prm[]: E, nu, sigma0, sigma_inf, delta, H, tol_g,
 * tol_step, max_iter.  The Newton iteration on the consistency condition
 * stops when |g| <= tol_g * sigma_y(alpha_n) (before an update) or when the
 * last update was at most tol_step in magnitude; more than max_iter updates
 * is a failure.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

int oracle_quadrature(int type, int tet_rule, double* pts, double* w);
int oracle_shape(int type, const double* p, double* N, double* dN);

#define J2_MAXN 8
#define J2_MAXQ 8

static int j2_nodes(int type) { return type == 0 ? 4 : type == 1 ? 5 : type == 2 ? 6 : 8; }

static double voce(const double* prm, double a) {
  return prm[2] + prm[5] * a + (prm[3] - prm[2]) * (1.0 - exp(-prm[4] * a));
}

static double voce_slope(const double* prm, double a) {
  return prm[5] + (prm[3] - prm[2]) * prm[4] * exp(-prm[4] * a);
}

/* ---------------------------------------------------------------------------
 * Radial return at one Gauss point.
 *
 *   elastic trial: e = eps - eps_p_n, s_tr = 2 mu dev(e), f = |s_tr| - sqrt(2/3) sigma_y(alpha_n)
 *   f <= 0: sigma = kappa tr(e) 1 + s_tr, D = kappa 1(x)1 + 2 mu I_dev (elastic)
 *   f > 0 : solve g(dg) = |s_tr| - 2 mu dg - sqrt(2/3) sigma_y(alpha_n + sqrt(2/3) dg) = 0
 *           by Newton from dg = 0 (g is convex and decreasing, so the iterates
 *           rise monotonically to the root), then with n = s_tr / |s_tr|:
 *           s = s_tr - 2 mu dg n,  eps_p = eps_p_n + dg n,  alpha = alpha_n + sqrt(2/3) dg
 *
 * Consistent tangent, from differentiating the update: with
 *   d|s_tr| = 2 mu n : d eps  and  d dg = n : d eps / (1 + sigma_y'(alpha) / (3 mu)),
 * ds = theta 2 mu I_dev d eps + |s_tr| d theta n gives
 *   D_ep = kappa 1(x)1 + 2 mu theta I_dev - 2 mu theta_bar n(x)n,
 *   theta = 1 - 2 mu dg / |s_tr|,  theta_bar = 1 / (1 + sigma_y'(alpha) / (3 mu)) - (1 - theta).
 *
 * eps, eps_p_n, eps_p, sig: tensor components (xx, yy, zz, xy, yz, xz);
 * D: 6x6 row-major acting on engineering strain.  Returns 0, or 1 when the
 * Newton iteration did not converge within max_iter updates.
 * ------------------------------------------------------------------------- */
static int j2_return(const double* prm, const double* eps, const double* eps_p_n, double alpha_n, double* sig,
                     double* D, double* eps_p, double* alpha, int* iters, int* yielded, double* thetas) {
  const double E = prm[0], nu = prm[1];
  const double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  const double mu = E / (2.0 * (1.0 + nu));
  const double kappa = lam + 2.0 * mu / 3.0;
  const double r23 = sqrt(2.0 / 3.0);
  double e[6];
  for (int i = 0; i < 6; ++i) e[i] = eps[i] - eps_p_n[i];
  const double tr = e[0] + e[1] + e[2];
  double s[6];
  for (int i = 0; i < 6; ++i) s[i] = 2.0 * mu * (e[i] - (i < 3 ? tr / 3.0 : 0.0));
  const double norm = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2] + 2.0 * (s[3] * s[3] + s[4] * s[4] + s[5] * s[5]));
  const double sy_n = voce(prm, alpha_n);
  const double f = norm - r23 * sy_n;

  double theta = 1.0, theta_bar = 0.0, nv[6] = {0, 0, 0, 0, 0, 0};
  double dg = 0.0;
  int it = 0;
  if (f <= 0.0) {
    for (int i = 0; i < 6; ++i) eps_p[i] = eps_p_n[i];
    *alpha = alpha_n;
    *yielded = 0;
  } else {
    const double tol_g = prm[6], tol_step = prm[7];
    const int max_iter = (int)prm[8];
    int ok = 0;
    for (;;) {
      const double a = alpha_n + r23 * dg;
      const double g = norm - 2.0 * mu * dg - r23 * voce(prm, a);
      if (fabs(g) <= tol_g * sy_n) { ok = 1; break; }
      if (it == max_iter) break;
      const double gp = -2.0 * mu - (2.0 / 3.0) * voce_slope(prm, a);
      const double step = -g / gp;
      dg += step;
      ++it;
      if (fabs(step) <= tol_step) { ok = 1; break; }
    }
    *iters = it;
    if (!ok) return 1;
    for (int i = 0; i < 6; ++i) nv[i] = s[i] / norm;
    const double a = alpha_n + r23 * dg;
    theta = 1.0 - 2.0 * mu * dg / norm;
    theta_bar = 1.0 / (1.0 + voce_slope(prm, a) / (3.0 * mu)) - (1.0 - theta);
    for (int i = 0; i < 6; ++i) {
      s[i] -= 2.0 * mu * dg * nv[i];
      eps_p[i] = eps_p_n[i] + dg * nv[i];
    }
    *alpha = a;
    *yielded = 1;
  }
  *iters = it;
  if (thetas) {
    thetas[0] = theta;
    thetas[1] = theta_bar;
  }
  for (int i = 0; i < 6; ++i) sig[i] = s[i] + (i < 3 ? kappa * tr : 0.0);
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      double v = 0.0;
      if (i < 3 && j < 3) v += kappa + 2.0 * mu * theta * ((i == j ? 1.0 : 0.0) - 1.0 / 3.0);
      if (i >= 3 && i == j) v += mu * theta;
      v -= 2.0 * mu * theta_bar * nv[i] * nv[j];
      D[6 * i + j] = v;
    }
  return 0;
}

int oracle_j2_point(const double* prm, const double* eps, const double* eps_p_n, double alpha_n, double* sig,
                    double* D, double* eps_p, double* alpha, int* iters, int* yielded) {
  return j2_return(prm, eps, eps_p_n, alpha_n, sig, D, eps_p, alpha, iters, yielded, NULL);
}

/* ---------------------------------------------------------------------------
 * Element tangent and internal force.  X, U: [nn][3] node coordinates and
 * displacements; state_n / state: [nq][7] (state_n NULL = virgin material);
 * iters, yielded: [nq] (may be NULL).  Ne / Nb (may be NULL): normwise error
 * scales |w detJ| (|lam'| + 2|mu'| + 2 mu |theta_bar|) |g_a| |g_b| and
 * |w detJ| |sigma|_F |g_a|, with lam' = kappa - 2 mu theta / 3 and
 * mu' = mu theta the isotropic part of D_ep.
 * Returns 0, 1 for det J <= 0, 2 for a return map that did not converge.
 * ------------------------------------------------------------------------- */
int oracle_j2_element(int type, const double* prm, const double* X, const double* U, const double* state_n,
                      double* Ae, double* be, double* Ne, double* Nb, double* state, int* iters, int* yielded) {
  const int nn = j2_nodes(type), n = 3 * nn;
  double pts[J2_MAXQ * 3], w[J2_MAXQ];
  const int nq = oracle_quadrature(type, 1, pts, w);
  memset(Ae, 0, sizeof(double) * n * n);
  memset(be, 0, sizeof(double) * n);
  if (Ne) memset(Ne, 0, sizeof(double) * n * n);
  if (Nb) memset(Nb, 0, sizeof(double) * n);
  const double E = prm[0], nu = prm[1];
  const double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  const double mu = E / (2.0 * (1.0 + nu));
  const double kappa = lam + 2.0 * mu / 3.0;
  for (int q = 0; q < nq; ++q) {
    double N[J2_MAXN], dN[J2_MAXN * 3];
    oracle_shape(type, pts + 3 * q, N, dN);
    double J[3][3] = {{0}};
    for (int a = 0; a < nn; ++a)
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) J[i][j] += X[3 * a + i] * dN[3 * a + j];
    double C[3][3];
    C[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    C[0][1] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    C[0][2] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    C[1][0] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    C[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    C[1][2] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    C[2][0] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    C[2][1] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    C[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    const double det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
    if (!(det > 0.0)) return 1;
    /* grad N_a = J^{-T} grad_xi N_a, (J^{-1})_{ji} = C_ij / det */
    double G[J2_MAXN][3], gn[J2_MAXN];
    for (int a = 0; a < nn; ++a) {
      for (int i = 0; i < 3; ++i) {
        G[a][i] = 0.0;
        for (int j = 0; j < 3; ++j) G[a][i] += dN[3 * a + j] * C[i][j] / det;
      }
      gn[a] = sqrt(G[a][0] * G[a][0] + G[a][1] * G[a][1] + G[a][2] * G[a][2]);
    }
    /* strain tensor components of sym(grad u) */
    double H[3][3] = {{0}};
    for (int a = 0; a < nn; ++a)
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) H[i][j] += U[3 * a + i] * G[a][j];
    const double eps[6] = {H[0][0], H[1][1], H[2][2], 0.5 * (H[0][1] + H[1][0]), 0.5 * (H[1][2] + H[2][1]),
                           0.5 * (H[0][2] + H[2][0])};
    static const double zero[7] = {0, 0, 0, 0, 0, 0, 0};
    const double* sn = state_n ? state_n + 7 * q : zero;
    double sig[6], D[36], ep[6], al, th[2];
    int it = 0, yl = 0;
    if (j2_return(prm, eps, sn, sn[6], sig, D, ep, &al, &it, &yl, th)) return 2;
    if (state) {
      for (int i = 0; i < 6; ++i) state[7 * q + i] = ep[i];
      state[7 * q + 6] = al;
    }
    if (iters) iters[q] = it;
    if (yielded) yielded[q] = yl;
    double B[J2_MAXN][6][3];
    memset(B, 0, sizeof(B));
    for (int a = 0; a < nn; ++a) {
      B[a][0][0] = G[a][0];
      B[a][1][1] = G[a][1];
      B[a][2][2] = G[a][2];
      B[a][3][0] = G[a][1]; B[a][3][1] = G[a][0];
      B[a][4][1] = G[a][2]; B[a][4][2] = G[a][1];
      B[a][5][0] = G[a][2]; B[a][5][2] = G[a][0];
    }
    const double wd = w[q] * det;
    const double theta = th[0], theta_bar = th[1];
    const double lam_p = kappa - 2.0 * mu * theta / 3.0, mu_iso = mu * theta;
    const double dscale = fabs(lam_p) + 2.0 * fabs(mu_iso) + 2.0 * mu * fabs(theta_bar);
    const double snorm =
        sqrt(sig[0] * sig[0] + sig[1] * sig[1] + sig[2] * sig[2] + 2.0 * (sig[3] * sig[3] + sig[4] * sig[4] + sig[5] * sig[5]));
    for (int a = 0; a < nn; ++a)
      for (int b = 0; b < nn; ++b)
        for (int c = 0; c < 3; ++c)
          for (int cc = 0; cc < 3; ++cc) {
            double s = 0.0;
            for (int I = 0; I < 6; ++I)
              for (int K = 0; K < 6; ++K) s += B[a][I][c] * D[6 * I + K] * B[b][K][cc];
            Ae[(3 * a + c) * n + 3 * b + cc] += wd * s;
            if (Ne) Ne[(3 * a + c) * n + 3 * b + cc] += fabs(wd) * dscale * gn[a] * gn[b];
          }
    /* f_int: B^T sigma with sigma in Voigt order (shear rows pair with engineering strain) */
    for (int a = 0; a < nn; ++a)
      for (int c = 0; c < 3; ++c) {
        double s = 0.0;
        for (int I = 0; I < 6; ++I) s += B[a][I][c] * sig[I];
        be[3 * a + c] += wd * s;
        if (Nb) Nb[3 * a + c] += fabs(wd) * snorm * gn[a];
      }
  }
  return 0;
}

/* ---------------------------------------------------------------------------
 * Full tangent + internal force assembly in element-index order, over the
 * oracle's own pattern (rp_s: scalar row_ptr, node_map: rank map), 3 dofs per
 * node.  U: [n_nodes][3].  state_n: [E][8][7] or NULL; state, iters, yielded:
 * [E][8][7], [E][8], [E][8] or NULL (slots past the rule's point count are left
 * untouched).  Returns 0, -(e+1) for an inverted element e, -(E+e+1) when the
 * return map of element e did not converge.
 * ------------------------------------------------------------------------- */
int64_t oracle_j2_assemble(int64_t n_nodes, int64_t n_elems, const uint8_t* types, const int64_t* conn_off,
                           const int32_t* conn, const double* coords, const double* prm, const double* U,
                           const double* state_n, const int64_t* rp_s, const int32_t* node_map, double* A,
                           double* b, double* NA, double* Nb, double* state, int32_t* iters, uint8_t* yielded) {
  (void)n_nodes;
  double X[3 * J2_MAXN], Ue[3 * J2_MAXN];
  double Ae[24 * 24], be[24], Ne[24 * 24], Nbe[24];
  int it[J2_MAXQ], yl[J2_MAXQ];
  int64_t off = 0;
  for (int64_t e = 0; e < n_elems; ++e) {
    const int ne = (int)(conn_off[e + 1] - conn_off[e]);
    const int32_t* en = conn + conn_off[e];
    for (int a = 0; a < ne; ++a)
      for (int i = 0; i < 3; ++i) {
        X[3 * a + i] = coords[3 * (int64_t)en[a] + i];
        Ue[3 * a + i] = U[3 * (int64_t)en[a] + i];
      }
    const int rc = oracle_j2_element(types[e], prm, X, Ue, state_n ? state_n + 56 * e : NULL, Ae, be, Ne, Nbe,
                                     state ? state + 56 * e : NULL, it, yl);
    if (rc == 1) return -(e + 1);
    if (rc == 2) return -(n_elems + e + 1);
    double pts[J2_MAXQ * 3], w[J2_MAXQ];
    const int nq = oracle_quadrature(types[e], 1, pts, w);
    for (int q = 0; q < nq; ++q) {
      if (iters) iters[8 * e + q] = it[q];
      if (yielded) yielded[8 * e + q] = (uint8_t)yl[q];
    }
    const int n = 3 * ne;
    for (int a = 0; a < ne; ++a)
      for (int c = 0; c < 3; ++c) {
        const int64_t row = 3 * (int64_t)en[a] + c;
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

/* ---------------------------------------------------------------------------
 * Gauss-point sweep without assembly (the element-wise loop; also the
 * load-amplitude fixture): the return map of every point of every element at
 * displacement scale*U, from state_n (NULL = virgin), writing the new state,
 * the stress [E][8][6], the Newton iteration counts and the yield flags
 * [E][8] (each may be NULL) and returning the number of points that yielded,
 * or -1 on an inverted element or a failed return map.
 * ------------------------------------------------------------------------- */
int64_t oracle_j2_sweep(int64_t n_elems, const uint8_t* types, const int64_t* conn_off, const int32_t* conn,
                        const double* coords, const double* prm, const double* U, double scale,
                        const double* state_n, double* state, double* stress, int32_t* iters, uint8_t* yielded) {
  int64_t count = 0;
  double X[3 * J2_MAXN], Ue[3 * J2_MAXN];
  for (int64_t e = 0; e < n_elems; ++e) {
    const int ne = (int)(conn_off[e + 1] - conn_off[e]);
    const int type = types[e];
    const int32_t* en = conn + conn_off[e];
    for (int a = 0; a < ne; ++a)
      for (int i = 0; i < 3; ++i) {
        X[3 * a + i] = coords[3 * (int64_t)en[a] + i];
        Ue[3 * a + i] = scale * U[3 * (int64_t)en[a] + i];
      }
    double pts[J2_MAXQ * 3], w[J2_MAXQ];
    const int nq = oracle_quadrature(type, 1, pts, w);
    for (int q = 0; q < nq; ++q) {
      double N[J2_MAXN], dN[J2_MAXN * 3];
      oracle_shape(type, pts + 3 * q, N, dN);
      double J[3][3] = {{0}};
      for (int a = 0; a < ne; ++a)
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) J[i][j] += X[3 * a + i] * dN[3 * a + j];
      double C[3][3];
      C[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
      C[0][1] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
      C[0][2] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
      C[1][0] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
      C[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
      C[1][2] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
      C[2][0] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
      C[2][1] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
      C[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
      const double det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
      if (!(det > 0.0)) return -1;
      double Hg[3][3] = {{0}};
      for (int a = 0; a < ne; ++a) {
        double g[3];
        for (int i = 0; i < 3; ++i) {
          g[i] = 0.0;
          for (int j = 0; j < 3; ++j) g[i] += dN[3 * a + j] * C[i][j] / det;
        }
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) Hg[i][j] += Ue[3 * a + i] * g[j];
      }
      const double eps[6] = {Hg[0][0], Hg[1][1], Hg[2][2], 0.5 * (Hg[0][1] + Hg[1][0]),
                             0.5 * (Hg[1][2] + Hg[2][1]), 0.5 * (Hg[0][2] + Hg[2][0])};
      static const double zero[7] = {0, 0, 0, 0, 0, 0, 0};
      const double* sn = state_n ? state_n + 56 * e + 7 * q : zero;
      double sig[6], D[36], ep[6], al;
      int it, yl;
      if (oracle_j2_point(prm, eps, sn, sn[6], sig, D, ep, &al, &it, &yl)) return -1;
      if (state) {
        for (int i = 0; i < 6; ++i) state[56 * e + 7 * q + i] = ep[i];
        state[56 * e + 7 * q + 6] = al;
      }
      if (stress)
        for (int i = 0; i < 6; ++i) stress[48 * e + 6 * q + i] = sig[i];
      if (iters) iters[8 * e + q] = it;
      if (yielded) yielded[8 * e + q] = (uint8_t)yl;
      count += yl;
    }
  }
  return count;
}
