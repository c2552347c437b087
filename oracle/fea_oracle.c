/*
 * fea_oracle.c -- plain, slow, single-threaded FP64 reference of finite
 * element assembly.  TEST INFRASTRUCTURE ONLY: it is called by the tests,
 * by the smoke check and by the CPU-baseline leg of the benchmark, never by
 * the engine.  It shares no code, header or table with the CUDA engine.
 *
 * What it computes (MPI+X assembly paper, Alg. "sequential assembly",
 * Sec. 2.1.1, and the local square matrices of Sec. 3.1):
 *
 *     for every element e, in element-index order:
 *         compute the element matrix A^e and right-hand side b^e by Gauss
 *         quadrature
 *         A += P_e^T A^e P_e,   b += P_e^T b^e
 *
 * into one CSR matrix whose pattern is "node i couples to node j iff some
 * element holds both" (diagonal included), rows sorted ascending, with d
 * interleaved dofs per node (dof = d*node + component).
 *
 * The paper gives the PDEs but no element formulation; the formulations
 * below are the textbook Galerkin ones (Hughes, "The Finite Element
 * Method", ch. 2-3; Zienkiewicz & Taylor vol. 1):
 *   diffusion : A^e_ab = sum_q w_q detJ_q k(x_q) grad N_a . grad N_b,
 *               b^e_a  = sum_q w_q detJ_q f N_a,      k(x) = k0 + k2 x^2
 *   elasticity: A^e_(a,c)(b,c') = sum_q w_q detJ_q (B_a^T D B_b)_(c,c'),
 *               b^e_(a,c) = sum_q w_q detJ_q f_c N_a,
 *               Voigt order (xx,yy,zz,xy,yz,xz), engineering shear, isotropic D.
 * Jacobian convention J_ij = dx_i/dxi_j; detJ <= 0 at a quadrature point is an
 * error (inverted element), never abs()-ed away.
 *
 * Alongside A and b it accumulates the magnitude sums S (same formula with
 * every factor replaced by its absolute value), the scale of the standard
 * a-priori floating point error bound used by the parity tests.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_TET4 0
#define OR_PYR5 1
#define OR_PRISM6 2
#define OR_HEX8 3

#define OR_OP_DIFFUSION 0
#define OR_OP_ELASTICITY 1

#define OR_MAXN 8
#define OR_MAXQ 8

static int or_nodes(int type) {
  switch (type) {
    case OR_TET4: return 4;
    case OR_PYR5: return 5;
    case OR_PRISM6: return 6;
    case OR_HEX8: return 8;
  }
  return -1;
}

/* ---------------------------------------------------------------------------
 * Reference shape functions N_a(xi) and derivatives dN_a/dxi_j.
 * ------------------------------------------------------------------------- */
static void or_shape(int type, const double p[3], double N[OR_MAXN], double dN[OR_MAXN][3]) {
  double x = p[0], y = p[1], z = p[2];
  if (type == OR_TET4) {
    /* linear simplex: N0 = 1-x-y-z, N1 = x, N2 = y, N3 = z */
    N[0] = 1.0 - x - y - z; N[1] = x; N[2] = y; N[3] = z;
    double d[4][3] = {{-1, -1, -1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    memcpy(dN, d, sizeof(d));
  } else if (type == OR_HEX8) {
    /* trilinear on [-1,1]^3, nodes (000,100,110,010,001,101,111,011) */
    static const double s[8][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
                                   {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};
    for (int a = 0; a < 8; ++a) {
      double fx = 1.0 + s[a][0] * x, fy = 1.0 + s[a][1] * y, fz = 1.0 + s[a][2] * z;
      N[a] = fx * fy * fz / 8.0;
      dN[a][0] = s[a][0] * fy * fz / 8.0;
      dN[a][1] = fx * s[a][1] * fz / 8.0;
      dN[a][2] = fx * fy * s[a][2] / 8.0;
    }
  } else if (type == OR_PRISM6) {
    /* linear triangle (L0 = 1-x-y, L1 = x, L2 = y) times linear in z on [-1,1] */
    double L[3] = {1.0 - x - y, x, y};
    double dL[3][2] = {{-1, -1}, {1, 0}, {0, 1}};
    for (int i = 0; i < 3; ++i) {
      double lo = 0.5 * (1.0 - z), hi = 0.5 * (1.0 + z);
      N[i] = L[i] * lo;
      N[i + 3] = L[i] * hi;
      dN[i][0] = dL[i][0] * lo;     dN[i][1] = dL[i][1] * lo;     dN[i][2] = -0.5 * L[i];
      dN[i + 3][0] = dL[i][0] * hi; dN[i + 3][1] = dL[i][1] * hi; dN[i + 3][2] = 0.5 * L[i];
    }
  } else { /* OR_PYR5 */
    /* rational 5-node pyramid (Bedrosian 1992): base [-1,1]^2 at z=0, apex (0,0,1).
     * base node i with signs (sx,sy): N = (1-z+sx x)(1-z+sy y) / (4(1-z)); apex N = z.
     * Only evaluated at interior points (z < 1). */
    static const double s[4][2] = {{-1, -1}, {1, -1}, {1, 1}, {-1, 1}};
    double D = 1.0 - z;
    for (int i = 0; i < 4; ++i) {
      double A = D + s[i][0] * x, B = D + s[i][1] * y;
      N[i] = A * B / (4.0 * D);
      dN[i][0] = s[i][0] * B / (4.0 * D);
      dN[i][1] = s[i][1] * A / (4.0 * D);
      dN[i][2] = (-(A + B) * D + A * B) / (4.0 * D * D);
    }
    N[4] = z;
    dN[4][0] = 0.0; dN[4][1] = 0.0; dN[4][2] = 1.0;
  }
}

/* ---------------------------------------------------------------------------
 * Quadrature rules.  tet_rule: 0 = 1-point centroid, 1 = 4-point degree 2.
 * hex 2x2x2 Gauss; prism 3-point triangle x 2-point Gauss; pyramid: Duffy
 * collapse of the cube, 2x2 Gauss-Legendre in the base times the 2-point
 * Gauss-Jacobi rule for the weight (1-t)^2 on t in [0,1].
 * ------------------------------------------------------------------------- */
static int or_quadrature(int type, int tet_rule, double pts[OR_MAXQ][3], double w[OR_MAXQ]) {
  const double g = 1.0 / sqrt(3.0);
  if (type == OR_TET4) {
    if (tet_rule == 0) {
      pts[0][0] = pts[0][1] = pts[0][2] = 0.25;
      w[0] = 1.0 / 6.0;
      return 1;
    }
    double a = (5.0 + 3.0 * sqrt(5.0)) / 20.0, b = (5.0 - sqrt(5.0)) / 20.0;
    double P[4][3] = {{b, b, b}, {a, b, b}, {b, a, b}, {b, b, a}};
    for (int q = 0; q < 4; ++q) {
      pts[q][0] = P[q][0]; pts[q][1] = P[q][1]; pts[q][2] = P[q][2];
      w[q] = 1.0 / 24.0;
    }
    return 4;
  }
  if (type == OR_HEX8) {
    int q = 0;
    for (int k = 0; k < 2; ++k)
      for (int j = 0; j < 2; ++j)
        for (int i = 0; i < 2; ++i) {
          pts[q][0] = i ? g : -g; pts[q][1] = j ? g : -g; pts[q][2] = k ? g : -g;
          w[q] = 1.0;
          ++q;
        }
    return 8;
  }
  if (type == OR_PRISM6) {
    double T[3][2] = {{1.0 / 6.0, 1.0 / 6.0}, {2.0 / 3.0, 1.0 / 6.0}, {1.0 / 6.0, 2.0 / 3.0}};
    int q = 0;
    for (int k = 0; k < 2; ++k)
      for (int t = 0; t < 3; ++t) {
        pts[q][0] = T[t][0]; pts[q][1] = T[t][1]; pts[q][2] = k ? g : -g;
        w[q] = 1.0 / 6.0;
        ++q;
      }
    return 6;
  }
  /* pyramid: t-nodes are the roots of t^2 - (2/3) t + 1/15 (orthogonal for (1-t)^2 on [0,1]);
   * weights from the moments m0 = 1/3, m1 = 1/12. */
  double r = sqrt(10.0) / 15.0;
  double t1 = 1.0 / 3.0 - r, t2 = 1.0 / 3.0 + r;
  double W2 = (1.0 / 12.0 - t1 / 3.0) / (t2 - t1);
  double W1 = 1.0 / 3.0 - W2;
  double tn[2] = {t1, t2}, tw[2] = {W1, W2};
  int q = 0;
  for (int k = 0; k < 2; ++k)
    for (int j = 0; j < 2; ++j)
      for (int i = 0; i < 2; ++i) {
        double u = i ? g : -g, v = j ? g : -g, t = tn[k];
        pts[q][0] = u * (1.0 - t); pts[q][1] = v * (1.0 - t); pts[q][2] = t;
        w[q] = tw[k];
        ++q;
      }
  return 8;
}

/* exported for the oracle's own tests */
int oracle_quadrature(int type, int tet_rule, double* pts, double* w) {
  double P[OR_MAXQ][3], W[OR_MAXQ];
  int nq = or_quadrature(type, tet_rule, P, W);
  for (int q = 0; q < nq; ++q) {
    pts[3 * q] = P[q][0]; pts[3 * q + 1] = P[q][1]; pts[3 * q + 2] = P[q][2];
    w[q] = W[q];
  }
  return nq;
}

int oracle_shape(int type, const double* p, double* N, double* dN) {
  double n[OR_MAXN], d[OR_MAXN][3];
  or_shape(type, p, n, d);
  int nn = or_nodes(type);
  for (int a = 0; a < nn; ++a) {
    N[a] = n[a];
    dN[3 * a] = d[a][0]; dN[3 * a + 1] = d[a][1]; dN[3 * a + 2] = d[a][2];
  }
  return nn;
}

/* ---------------------------------------------------------------------------
 * Element matrix.  params: diffusion {k0, k2, f}; elasticity {E, nu, fx, fy, fz}.
 * Ae is (nn*d) x (nn*d) row-major with index a*d+c, be has nn*d entries, Se/Sb
 * the componentwise magnitude sums.  Ne (may be NULL) receives the normwise
 * scale of each entry: the Cauchy-Schwarz bound of every quadrature term,
 * |w detJ| |k| |g_a| |g_b| (diffusion) or |w detJ| (|lam| + 2|mu|) |g_a| |g_b|
 * (elasticity), with g_a = grad N_a and |.| the Euclidean norm.  A rounding of
 * the gradients by a relative amount eps (normwise) moves an entry by at most
 * about eps times its normwise scale.
 * Returns 0, or 1 if detJ <= 0 at some quadrature point.
 * ------------------------------------------------------------------------- */
int oracle_element(int type, int tet_rule, int op, const double* params, const double* X,
                   double* Ae, double* be, double* Se, double* Sb, double* Ne) {
  int nn = or_nodes(type);
  int d = (op == OR_OP_DIFFUSION) ? 1 : 3;
  int n = nn * d;
  double pts[OR_MAXQ][3], w[OR_MAXQ];
  int nq = or_quadrature(type, tet_rule, pts, w);
  memset(Ae, 0, sizeof(double) * n * n);
  memset(be, 0, sizeof(double) * n);
  memset(Se, 0, sizeof(double) * n * n);
  memset(Sb, 0, sizeof(double) * n);
  if (Ne) memset(Ne, 0, sizeof(double) * n * n);

  double D[6][6];
  double lam = 0.0, mu = 0.0;
  memset(D, 0, sizeof(D));
  if (op == OR_OP_ELASTICITY) {
    double E = params[0], nu = params[1];
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    mu = E / (2.0 * (1.0 + nu));
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j) D[i][j] = lam;
      D[i][i] = lam + 2.0 * mu;
      D[i + 3][i + 3] = mu;
    }
  }

  for (int q = 0; q < nq; ++q) {
    double N[OR_MAXN], dN[OR_MAXN][3];
    or_shape(type, pts[q], N, dN);
    /* J_ij = dx_i/dxi_j */
    double J[3][3] = {{0}};
    double xq[3] = {0, 0, 0};
    for (int a = 0; a < nn; ++a)
      for (int i = 0; i < 3; ++i) {
        xq[i] += N[a] * X[3 * a + i];
        for (int j = 0; j < 3; ++j) J[i][j] += X[3 * a + i] * dN[a][j];
      }
    /* inverse by the adjugate */
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
    double det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
    if (!(det > 0.0)) return 1;
    double Jinv[3][3]; /* Jinv[j][i] = C[i][j] / det */
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) Jinv[j][i] = C[i][j] / det;
    /* grad N_a: dN_a/dx_i = sum_j dN_a/dxi_j (J^{-1})_{j i} */
    double G[OR_MAXN][3];
    for (int a = 0; a < nn; ++a)
      for (int i = 0; i < 3; ++i) {
        G[a][i] = 0.0;
        for (int j = 0; j < 3; ++j) G[a][i] += dN[a][j] * Jinv[j][i];
      }
    double wd = w[q] * det;
    double gnorm[OR_MAXN];
    for (int a = 0; a < nn; ++a) gnorm[a] = sqrt(G[a][0] * G[a][0] + G[a][1] * G[a][1] + G[a][2] * G[a][2]);

    if (op == OR_OP_DIFFUSION) {
      double k0 = params[0], k2 = params[1], f = params[2];
      double k = k0 + k2 * xq[0] * xq[0];
      double kabs = fabs(k0) + fabs(k2) * xq[0] * xq[0];
      for (int a = 0; a < nn; ++a) {
        for (int b = 0; b < nn; ++b) {
          double s = 0.0, sa = 0.0;
          for (int i = 0; i < 3; ++i) { s += G[a][i] * G[b][i]; sa += fabs(G[a][i] * G[b][i]); }
          Ae[a * n + b] += wd * k * s;
          Se[a * n + b] += fabs(wd) * kabs * sa;
          if (Ne) Ne[a * n + b] += fabs(wd) * kabs * gnorm[a] * gnorm[b];
        }
        be[a] += wd * f * N[a];
        Sb[a] += fabs(wd) * fabs(f) * fabs(N[a]);
      }
    } else {
      /* B_a (6x3): rows xx,yy,zz,xy,yz,xz */
      double B[OR_MAXN][6][3];
      memset(B, 0, sizeof(B));
      for (int a = 0; a < nn; ++a) {
        B[a][0][0] = G[a][0];
        B[a][1][1] = G[a][1];
        B[a][2][2] = G[a][2];
        B[a][3][0] = G[a][1]; B[a][3][1] = G[a][0];
        B[a][4][1] = G[a][2]; B[a][4][2] = G[a][1];
        B[a][5][0] = G[a][2]; B[a][5][2] = G[a][0];
      }
      for (int a = 0; a < nn; ++a)
        for (int b = 0; b < nn; ++b)
          for (int c = 0; c < 3; ++c)
            for (int cc = 0; cc < 3; ++cc) {
              double s = 0.0, sa = 0.0;
              for (int I = 0; I < 6; ++I)
                for (int K = 0; K < 6; ++K) {
                  double t = B[a][I][c] * D[I][K] * B[b][K][cc];
                  s += t;
                  sa += fabs(t);
                }
              Ae[(a * 3 + c) * n + b * 3 + cc] += wd * s;
              Se[(a * 3 + c) * n + b * 3 + cc] += fabs(wd) * sa;
              if (Ne)
                Ne[(a * 3 + c) * n + b * 3 + cc] += fabs(wd) * (fabs(lam) + 2.0 * fabs(mu)) * gnorm[a] * gnorm[b];
            }
      for (int a = 0; a < nn; ++a)
        for (int c = 0; c < 3; ++c) {
          be[a * 3 + c] += wd * params[2 + c] * N[a];
          Sb[a * 3 + c] += fabs(wd) * fabs(params[2 + c]) * fabs(N[a]);
        }
    }
  }
  return 0;
}

/* ---------------------------------------------------------------------------
 * Pattern: node i couples to node j iff an element holds both.
 * Row i = sorted unique union of the nodes of the elements incident to i.
 * Two-call protocol: col_idx == NULL -> fill row_ptr only, return nnz.
 * node_map[map_off(e) + a*n_e + b] = rank of conn[e][b] in row conn[e][a]
 * (map_off(e) = sum over e' < e of n_e'^2).
 * Returns nnz, or -1 on bad input.
 * ------------------------------------------------------------------------- */
static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

int64_t oracle_pattern(int64_t n_nodes, int64_t n_elems, const uint8_t* types, const int64_t* conn_off,
                       const int32_t* conn, int64_t* row_ptr, int32_t* col_idx, int32_t* node_map) {
  if (n_nodes <= 0 || n_elems < 0) return -1;
  /* node -> incident elements */
  int64_t* cnt = (int64_t*)calloc((size_t)n_nodes + 1, sizeof(int64_t));
  for (int64_t e = 0; e < n_elems; ++e) {
    if (or_nodes(types[e]) != conn_off[e + 1] - conn_off[e]) { free(cnt); return -1; }
    for (int64_t t = conn_off[e]; t < conn_off[e + 1]; ++t) {
      if (conn[t] < 0 || conn[t] >= n_nodes) { free(cnt); return -1; }
      cnt[conn[t] + 1]++;
    }
  }
  for (int64_t i = 0; i < n_nodes; ++i) cnt[i + 1] += cnt[i];
  int64_t* inc = (int64_t*)malloc(sizeof(int64_t) * (size_t)(cnt[n_nodes] + 1));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_nodes + 1));
  memcpy(fill, cnt, sizeof(int64_t) * (size_t)n_nodes);
  for (int64_t e = 0; e < n_elems; ++e)
    for (int64_t t = conn_off[e]; t < conn_off[e + 1]; ++t) inc[fill[conn[t]]++] = e;

  int32_t* buf = NULL;
  int64_t bufcap = 0;
  row_ptr[0] = 0;
  for (int64_t i = 0; i < n_nodes; ++i) {
    int64_t m = 0;
    for (int64_t t = cnt[i]; t < cnt[i + 1]; ++t) m += conn_off[inc[t] + 1] - conn_off[inc[t]];
    if (m > bufcap) { bufcap = 2 * m + 16; buf = (int32_t*)realloc(buf, sizeof(int32_t) * (size_t)bufcap); }
    m = 0;
    for (int64_t t = cnt[i]; t < cnt[i + 1]; ++t) {
      int64_t e = inc[t];
      for (int64_t u = conn_off[e]; u < conn_off[e + 1]; ++u) buf[m++] = conn[u];
    }
    qsort(buf, (size_t)m, sizeof(int32_t), cmp_i32);
    int64_t k = 0;
    for (int64_t u = 0; u < m; ++u)
      if (u == 0 || buf[u] != buf[u - 1]) buf[k++] = buf[u];
    if (col_idx) memcpy(col_idx + row_ptr[i], buf, sizeof(int32_t) * (size_t)k);
    row_ptr[i + 1] = row_ptr[i] + k;
  }
  if (col_idx && node_map) {
    int64_t off = 0;
    for (int64_t e = 0; e < n_elems; ++e) {
      int64_t ne = conn_off[e + 1] - conn_off[e];
      for (int64_t a = 0; a < ne; ++a) {
        int32_t i = conn[conn_off[e] + a];
        const int32_t* row = col_idx + row_ptr[i];
        int64_t len = row_ptr[i + 1] - row_ptr[i];
        for (int64_t b = 0; b < ne; ++b) {
          int32_t j = conn[conn_off[e] + b];
          const int32_t* hit = (const int32_t*)bsearch(&j, row, (size_t)len, sizeof(int32_t), cmp_i32);
          node_map[off + a * ne + b] = (int32_t)(hit - row);
        }
      }
      off += ne * ne;
    }
  }
  int64_t nnz = row_ptr[n_nodes];
  free(buf); free(inc); free(fill); free(cnt);
  return nnz;
}

/* Scalar expansion with d interleaved dofs: row d*i+c holds columns d*j+c'
 * for the node neighbours j in order. */
void oracle_expand_pattern(int64_t n_nodes, int d, const int64_t* rp, const int32_t* col,
                           int64_t* rp_s, int32_t* col_s) {
  rp_s[0] = 0;
  for (int64_t i = 0; i < n_nodes; ++i) {
    int64_t deg = rp[i + 1] - rp[i];
    for (int c = 0; c < d; ++c) {
      int64_t r = d * i + c;
      for (int64_t k = 0; k < deg; ++k)
        for (int cc = 0; cc < d; ++cc) col_s[rp_s[r] + d * k + cc] = d * col[rp[i] + k] + cc;
      rp_s[r + 1] = rp_s[r] + d * deg;
    }
  }
}

/* ---------------------------------------------------------------------------
 * Full assembly in element-index order (Alg. "sequential assembly").
 * rp_s/node_map: the oracle's own pattern (scalar row_ptr + rank map).
 * Returns 0, or -(e+1) for the first inverted element e.
 * ------------------------------------------------------------------------- */
int64_t oracle_assemble(int64_t n_nodes, int64_t n_elems, const uint8_t* types, const int64_t* conn_off,
                        const int32_t* conn, const double* coords, int op, int tet_rule,
                        const double* params, const int64_t* rp_s, const int32_t* node_map,
                        double* A, double* b, double* SA, double* Sb, double* NA) {
  int d = (op == OR_OP_DIFFUSION) ? 1 : 3;
  (void)n_nodes;
  double X[3 * OR_MAXN];
  double Ae[24 * 24], be[24], Se[24 * 24], Sbe[24], Ne[24 * 24];
  int64_t off = 0;
  for (int64_t e = 0; e < n_elems; ++e) {
    int ne = (int)(conn_off[e + 1] - conn_off[e]);
    const int32_t* en = conn + conn_off[e];
    for (int a = 0; a < ne; ++a)
      for (int i = 0; i < 3; ++i) X[3 * a + i] = coords[3 * (int64_t)en[a] + i];
    if (oracle_element(types[e], tet_rule, op, params, X, Ae, be, Se, Sbe, Ne)) return -(e + 1);
    int n = ne * d;
    for (int a = 0; a < ne; ++a)
      for (int c = 0; c < d; ++c) {
        int64_t row = d * (int64_t)en[a] + c;
        for (int bb = 0; bb < ne; ++bb) {
          int64_t k = node_map[off + a * ne + bb];
          for (int cc = 0; cc < d; ++cc) {
            int64_t pos = rp_s[row] + d * k + cc;
            A[pos] += Ae[(a * d + c) * n + bb * d + cc];
            if (SA) SA[pos] += Se[(a * d + c) * n + bb * d + cc];
            if (NA) NA[pos] += Ne[(a * d + c) * n + bb * d + cc];
          }
        }
        b[row] += be[a * d + c];
        if (Sb) Sb[row] += Sbe[a * d + c];
      }
    off += (int64_t)ne * ne;
  }
  return 0;
}

/* ---------------------------------------------------------------------------
 * Rows of the assembled system for a few requested nodes (all d rows each),
 * summed over all elements in element-index order -- the same definition as
 * oracle_assemble restricted to those rows, for sampled checks of meshes too
 * large for a full oracle run.  Output per requested node r: its columns are
 * the sorted unique neighbours (computed here); values are written to
 * vals[r*max_cols*d*d ...] as d rows of (deg*d) entries; cols_out[r*max_cols + k]
 * gets the node neighbours, deg_out[r] the degree.  Returns 0, -(e+1) for an
 * inverted element, or -1 when a row has more than max_cols neighbours.
 * ------------------------------------------------------------------------- */
int64_t oracle_assemble_rows(int64_t n_nodes, int64_t n_elems, const uint8_t* types, const int64_t* conn_off,
                             const int32_t* conn, const double* coords, int op, int tet_rule,
                             const double* params, int64_t n_req, const int32_t* req_nodes, int64_t max_cols,
                             int32_t* cols_out, int64_t* deg_out, double* vals, double* svals,
                             double* bvals, double* sbvals, double* nvals) {
  int d = (op == OR_OP_DIFFUSION) ? 1 : 3;
  int64_t* slot = (int64_t*)malloc(sizeof(int64_t) * (size_t)n_nodes);
  for (int64_t i = 0; i < n_nodes; ++i) slot[i] = -1;
  for (int64_t r = 0; r < n_req; ++r) { slot[req_nodes[r]] = r; deg_out[r] = 0; }
  /* pass 1: neighbour lists of the requested rows */
  int32_t* tmp = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_req * max_cols * 8 + 8));
  int64_t* tcount = (int64_t*)calloc((size_t)n_req, sizeof(int64_t));
  for (int64_t e = 0; e < n_elems; ++e) {
    int ne = (int)(conn_off[e + 1] - conn_off[e]);
    const int32_t* en = conn + conn_off[e];
    for (int a = 0; a < ne; ++a) {
      int64_t r = slot[en[a]];
      if (r < 0) continue;
      for (int bb = 0; bb < ne; ++bb) {
        if (tcount[r] >= max_cols * 8) { free(slot); free(tmp); free(tcount); return -1; }
        tmp[r * max_cols * 8 + tcount[r]++] = en[bb];
      }
    }
  }
  for (int64_t r = 0; r < n_req; ++r) {
    int32_t* t = tmp + r * max_cols * 8;
    qsort(t, (size_t)tcount[r], sizeof(int32_t), cmp_i32);
    int64_t k = 0;
    for (int64_t u = 0; u < tcount[r]; ++u)
      if (u == 0 || t[u] != t[u - 1]) {
        if (k >= max_cols) { free(slot); free(tmp); free(tcount); return -1; }
        cols_out[r * max_cols + k++] = t[u];
      }
    deg_out[r] = k;
  }
  memset(vals, 0, sizeof(double) * (size_t)(n_req * max_cols * d * d));
  memset(svals, 0, sizeof(double) * (size_t)(n_req * max_cols * d * d));
  memset(nvals, 0, sizeof(double) * (size_t)(n_req * max_cols * d * d));
  memset(bvals, 0, sizeof(double) * (size_t)(n_req * d));
  memset(sbvals, 0, sizeof(double) * (size_t)(n_req * d));
  double X[3 * OR_MAXN];
  double Ae[24 * 24], be[24], Se[24 * 24], Sbe[24], Ne[24 * 24];
  for (int64_t e = 0; e < n_elems; ++e) {
    int ne = (int)(conn_off[e + 1] - conn_off[e]);
    const int32_t* en = conn + conn_off[e];
    int hit = 0;
    for (int a = 0; a < ne; ++a) hit |= slot[en[a]] >= 0;
    if (!hit) continue;
    for (int a = 0; a < ne; ++a)
      for (int i = 0; i < 3; ++i) X[3 * a + i] = coords[3 * (int64_t)en[a] + i];
    if (oracle_element(types[e], tet_rule, op, params, X, Ae, be, Se, Sbe, Ne)) {
      free(slot); free(tmp); free(tcount); return -(e + 1);
    }
    int n = ne * d;
    for (int a = 0; a < ne; ++a) {
      int64_t r = slot[en[a]];
      if (r < 0) continue;
      const int32_t* row = cols_out + r * max_cols;
      for (int bb = 0; bb < ne; ++bb) {
        const int32_t* h = (const int32_t*)bsearch(&en[bb], row, (size_t)deg_out[r], sizeof(int32_t), cmp_i32);
        int64_t k = h - row;
        for (int c = 0; c < d; ++c)
          for (int cc = 0; cc < d; ++cc) {
            int64_t pos = r * max_cols * d * d + c * (deg_out[r] * d) + d * k + cc;
            vals[pos] += Ae[(a * d + c) * n + bb * d + cc];
            svals[pos] += Se[(a * d + c) * n + bb * d + cc];
            nvals[pos] += Ne[(a * d + c) * n + bb * d + cc];
          }
      }
      for (int c = 0; c < d; ++c) {
        bvals[r * d + c] += be[a * d + c];
        sbvals[r * d + c] += Sbe[a * d + c];
      }
    }
  }
  free(slot); free(tmp); free(tcount);
  return 0;
}
