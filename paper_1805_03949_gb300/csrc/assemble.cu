// assemble.cu -- batched element integration and race-free scatter into CSR.
//
// The element loop of the MPI+X assembly paper (Alg. "sequential
// assembly", Sec. 2.1.1) on the GPU: every CTA integrates a tile of elements
// of one type and adds the element matrices into A and b.  The race on the
// shared entries (Sec. 3.2.1) is treated by the variant of fea_scatter:
//   ATOMIC  FP64 atomic adds, the GPU form of Alg. "no coloring".
//
// Tile schedule of one CTA (128 threads, EPC elements):
//   phase 0  gather the node coordinates of the tile into shared memory
//   phase 1  one thread per (element, quadrature point): Jacobian, det, J^{-1},
//            physical gradients g_a and the weight w*detJ (FP64, or FP32 with
//            an FP64 redo of distorted elements)
//   phase 2  LPE = n_e * SPLIT lanes per element: lane (a, half) accumulates
//            the row block A^e_(a, b) for its NB columns b over the points
//   phase 3  the same lane scatters its row block through the rank map.
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "element.cuh"
#include "fea_internal.cuh"
#include "sched.cuh"

namespace fea {

// ---------------------------------------------------------------------------
// host: reference tables
// ---------------------------------------------------------------------------
static void ref_shape(int type, const double p[3], double N[8], double dN[8][3]) {
  const double x = p[0], y = p[1], z = p[2];
  for (int a = 0; a < 8; ++a) N[a] = dN[a][0] = dN[a][1] = dN[a][2] = 0.0;
  switch (type) {
    case FEA_TET4: {
      N[0] = 1.0 - x - y - z;
      N[1] = x;
      N[2] = y;
      N[3] = z;
      for (int j = 0; j < 3; ++j) {
        dN[0][j] = -1.0;
        dN[j + 1][j] = 1.0;
      }
      break;
    }
    case FEA_HEX8: {
      // corner signs in (000,100,110,010,001,101,111,011) order
      for (int a = 0; a < 8; ++a) {
        const int bx = ((a + 1) >> 1) & 1, by = (a >> 1) & 1, bz = a >> 2;
        const double sx = bx ? 1.0 : -1.0, sy = by ? 1.0 : -1.0, sz = bz ? 1.0 : -1.0;
        const double fx = 0.5 * (1.0 + sx * x), fy = 0.5 * (1.0 + sy * y), fz = 0.5 * (1.0 + sz * z);
        N[a] = fx * fy * fz;
        dN[a][0] = 0.5 * sx * fy * fz;
        dN[a][1] = 0.5 * sy * fx * fz;
        dN[a][2] = 0.5 * sz * fx * fy;
      }
      break;
    }
    case FEA_PRISM6: {
      const double L[3] = {1.0 - x - y, x, y};
      const double Lx[3] = {-1.0, 1.0, 0.0}, Ly[3] = {-1.0, 0.0, 1.0};
      for (int s = 0; s < 2; ++s) {
        const double h = 0.5 * (1.0 + (s ? z : -z)), hz = s ? 0.5 : -0.5;
        for (int i = 0; i < 3; ++i) {
          N[3 * s + i] = L[i] * h;
          dN[3 * s + i][0] = Lx[i] * h;
          dN[3 * s + i][1] = Ly[i] * h;
          dN[3 * s + i][2] = L[i] * hz;
        }
      }
      break;
    }
    case FEA_PYR5: {
      // base corner i: N = (1 - z + sx x)(1 - z + sy y) / (4 (1 - z)); apex: N = z
      const double sx[4] = {-1.0, 1.0, 1.0, -1.0}, sy[4] = {-1.0, -1.0, 1.0, 1.0};
      const double t = 1.0 - z;
      for (int i = 0; i < 4; ++i) {
        const double u = t + sx[i] * x, v = t + sy[i] * y;
        N[i] = u * v / (4.0 * t);
        dN[i][0] = sx[i] * v / (4.0 * t);
        dN[i][1] = sy[i] * u / (4.0 * t);
        // d/dz of u v / (4 t) with du/dz = dv/dz = -1, dt/dz = -1
        dN[i][2] = (u * v - t * (u + v)) / (4.0 * t * t);
      }
      N[4] = z;
      dN[4][2] = 1.0;
      break;
    }
  }
}

static int ref_points(int slot, double P[8][3], double W[8]) {
  const double g = 1.0 / std::sqrt(3.0);
  const double gp[2] = {-g, g};
  switch (slot) {
    case kRuleTet1:
      P[0][0] = P[0][1] = P[0][2] = 0.25;
      W[0] = 1.0 / 6.0;
      return 1;
    case kRuleTet4: {
      const double a = (5.0 + 3.0 * std::sqrt(5.0)) / 20.0, b = (5.0 - std::sqrt(5.0)) / 20.0;
      for (int q = 0; q < 4; ++q) {
        for (int j = 0; j < 3; ++j) P[q][j] = (q == j + 1) ? a : b;
        W[q] = 1.0 / 24.0;
      }
      return 4;
    }
    case kRulePrism6: {
      const double tri[3][2] = {{1.0 / 6.0, 1.0 / 6.0}, {2.0 / 3.0, 1.0 / 6.0}, {1.0 / 6.0, 2.0 / 3.0}};
      for (int q = 0; q < 6; ++q) {
        P[q][0] = tri[q % 3][0];
        P[q][1] = tri[q % 3][1];
        P[q][2] = gp[q / 3];
        W[q] = 1.0 / 6.0;
      }
      return 6;
    }
    case kRuleHex8:
      for (int q = 0; q < 8; ++q) {
        P[q][0] = gp[q & 1];
        P[q][1] = gp[(q >> 1) & 1];
        P[q][2] = gp[q >> 2];
        W[q] = 1.0;
      }
      return 8;
    default: {  // pyramid: collapsed cube, 2x2 Gauss x Gauss-Jacobi (weight (1-t)^2 on [0,1])
      const double r = std::sqrt(10.0) / 15.0;
      const double t[2] = {1.0 / 3.0 - r, 1.0 / 3.0 + r};
      const double w2 = (1.0 / 12.0 - t[0] / 3.0) / (t[1] - t[0]);
      const double wt[2] = {1.0 / 3.0 - w2, w2};
      for (int q = 0; q < 8; ++q) {
        const int k = q >> 2;
        P[q][0] = gp[q & 1] * (1.0 - t[k]);
        P[q][1] = gp[(q >> 1) & 1] * (1.0 - t[k]);
        P[q][2] = t[k];
        W[q] = wt[k];
      }
      return 8;
    }
  }
}

const RefRule& host_rule(int slot) {
  static RefRule rules[kNumRules];
  static std::once_flag once;
  std::call_once(once, [] {
    for (int s = 0; s < kNumRules; ++s) {
      RefRule& R = rules[s];
      std::memset(&R, 0, sizeof(R));
      double P[8][3], W[8];
      const int nq = ref_points(s, P, W);
      for (int q = 0; q < nq; ++q) {
        double N[8], dN[8][3];
        ref_shape(rule_type(s), P[q], N, dN);
        R.w[q] = W[q];
        R.wf[q] = (float)W[q];
        for (int a = 0; a < 8; ++a) {
          R.N[q][a] = N[a];
          R.Nf[q][a] = (float)N[a];
          for (int j = 0; j < 3; ++j) {
            R.dN[q][a][j] = dN[a][j];
            R.dNf[q][a][j] = (float)dN[a][j];
          }
        }
      }
    }
  });
  return rules[slot];
}

// ---------------------------------------------------------------------------
// device
// ---------------------------------------------------------------------------
struct AsmParams {
  const double* coords;
  const int32_t* tconn;     // [n][NN] packed connectivity of the group
  const int32_t* ids;       // [n] original element ids (nullptr: identity)
  const int64_t* mapoff;    // [n] node_map offsets (nullptr: id * NN^2)
  const int32_t* list;      // launch index -> index in the group (nullptr: identity; coloring)
  int64_t n;                // elements of this launch
  const int64_t* row_ptr;
  const int32_t* node_map;
  double* A;
  double* b;
  DevStatus* st;
  double k0, k2, src;       // diffusion
  double lam, mu;           // elasticity
  double f[3];
  int geo64;                // FP32 tiles: 1 = FP64 geometry for every element, 0 = adaptive
};

__device__ __forceinline__ int64_t group_index(const AsmParams& P, int64_t et) {
  return P.list ? (int64_t)P.list[et] : et;
}
__device__ __forceinline__ int64_t original_id(const AsmParams& P, int64_t et) {
  const int64_t g = group_index(P, et);
  return P.ids ? (int64_t)P.ids[g] : g;
}

template <int OP, int PREC, int NN, int NQ, int EPC>
struct TileSmem {
  using R = typename std::conditional<PREC == FEA_FP64, double, float>::type;
  double X[EPC][NN][3];     // node coordinates
  R G[EPC][NQ][NN][3];      // physical gradients
  R S[EPC][NQ];             // w detJ k(x_q)
  R W[EPC][NQ];             // w detJ
  int flag[EPC];            // FP32 mode: element is distorted -> FP64 geometry
};

// Tile values of point q from the FP64 Jacobian J' = s J (s a power of two):
// det J = det'/s^3, grad N_a = J^{-T} grad_xi N_a = s C' grad_xi N_a / det'.
// FP64 tiles keep FP64; FP32 tiles round the cofactors and the determinant
// once and form the gradients in FP32.
// (the point's values from the cofactors C' and det' of J' = s J)
template <int OP, int NN, typename Smem>
__device__ __forceinline__ void geometry_store(Smem& sm, const RefRule& rr, int le, int q, const double (&C)[3][3],
                                               double det, double s, double xq, const AsmParams& P) {
  using R = std::remove_reference_t<decltype(sm.G[0][0][0][0])>;
  if constexpr (std::is_same<R, double>::value) {
    const double wd = rr.w[q] * det * (1.0 / (s * s * s));
    const double inv = s / det;
#pragma unroll
    for (int a = 0; a < NN; ++a)
#pragma unroll
      for (int i = 0; i < 3; ++i)
        // g_a,i = sum_j dN_a/dxi_j (J^{-1})_{j i},  (J^{-1})_{j i} = C_{i j} / det
        sm.G[le][q][a][i] = (rr.dN[q][a][0] * C[i][0] + rr.dN[q][a][1] * C[i][1] + rr.dN[q][a][2] * C[i][2]) * inv;
    sm.W[le][q] = wd;
    if constexpr (OP == FEA_OP_DIFFUSION)
      sm.S[le][q] = wd * (P.k0 + P.k2 * xq * xq);
    else
      sm.S[le][q] = wd;
  } else {
    float Cf[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) Cf[i][j] = f64_to_f32_rn(C[i][j]);
    const float detf = f64_to_f32_rn(det);
    const float inv = (float)s / detf;
#pragma unroll
    for (int a = 0; a < NN; ++a)
#pragma unroll
      for (int i = 0; i < 3; ++i)
        sm.G[le][q][a][i] = (rr.dNf[q][a][0] * Cf[i][0] + rr.dNf[q][a][1] * Cf[i][1] + rr.dNf[q][a][2] * Cf[i][2]) * inv;
    const float wdf = rr.wf[q] * detf * (float)(1.0 / (s * s * s));
    sm.W[le][q] = wdf;
    if constexpr (OP == FEA_OP_DIFFUSION) {
      const float x = f64_to_f32_rn(xq);
      sm.S[le][q] = wdf * (f64_to_f32_rn(P.k0) + f64_to_f32_rn(P.k2) * x * x);
    } else {
      sm.S[le][q] = wdf;
    }
  }
}

template <int OP, int NN, typename Smem>
__device__ __forceinline__ void geometry_finish(Smem& sm, const RefRule& rr, int le, int q, int64_t elem_id,
                                                double (&J)[3][3], double s, double xq, const AsmParams& P) {
  double C[3][3];
  cofactors(J, C);
  const double det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
  if (!(det > 0.0)) latch_error(P.st, FEA_ERR_INVERTED_ELEMENT, (unsigned long long)elem_id);
  geometry_store<OP, NN>(sm, rr, le, q, C, det, s, xq, P);
}

// FP64 geometry of point q of element le, J from the node coordinates (REL:
// nodes 1 .. NN-1 hold their differences to node 0 already)
template <int OP, int NN, bool REL = false, typename Smem>
__device__ __forceinline__ void geometry_fp64(Smem& sm, const RefRule& rr, int le, int q, int64_t elem_id,
                                              const AsmParams& P) {
  double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  double xq = sm.X[le][0][0];
#pragma unroll
  for (int a = 1; a < NN; ++a) {
    const double d0 = REL ? sm.X[le][a][0] : sm.X[le][a][0] - sm.X[le][0][0];
    const double d1 = REL ? sm.X[le][a][1] : sm.X[le][a][1] - sm.X[le][0][1];
    const double d2 = REL ? sm.X[le][a][2] : sm.X[le][a][2] - sm.X[le][0][2];
    xq += rr.N[q][a] * d0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      J[0][j] += d0 * rr.dN[q][a][j];
      J[1][j] += d1 * rr.dN[q][a][j];
      J[2][j] += d2 * rr.dN[q][a][j];
    }
  }
  geometry_finish<OP, NN>(sm, rr, le, q, elem_id, J, 1.0, xq, P);
}

// FP32 geometry on coordinates relative to node 0; returns false when the
// element must take the FP64 path (distorted: Frobenius condition number of J
// above FEA_KAPPA_FP64, or a determinant FP32 cannot trust).
template <int OP, int NN, typename Smem>
__device__ __forceinline__ bool geometry_fp32(Smem& sm, const RefRule& rr, int le, int q, const AsmParams& P) {
  float J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  float xr = 0.0f;
#pragma unroll
  for (int a = 1; a < NN; ++a) {
    const float d0 = f64_to_f32_rn(sm.X[le][a][0] - sm.X[le][0][0]);
    const float d1 = f64_to_f32_rn(sm.X[le][a][1] - sm.X[le][0][1]);
    const float d2 = f64_to_f32_rn(sm.X[le][a][2] - sm.X[le][0][2]);
    xr += rr.Nf[q][a] * d0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      J[0][j] += d0 * rr.dNf[q][a][j];
      J[1][j] += d1 * rr.dNf[q][a][j];
      J[2][j] += d2 * rr.dNf[q][a][j];
    }
  }
  float C[3][3];
  cofactors(J, C);
  const float det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
  float nj = 0.0f, nc = 0.0f;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      nj += J[i][j] * J[i][j];
      nc += C[i][j] * C[i][j];
    }
  // kappa_F^2 = |J|_F^2 |J^{-1}|_F^2 = |J|_F^2 |C|_F^2 / det^2
  const float kappa2_max = (float)(FEA_KAPPA_FP64 * FEA_KAPPA_FP64);
  if (!(det > 0.0f) || !(nj * nc <= kappa2_max * det * det)) return false;
  const float inv = 1.0f / det;
#pragma unroll
  for (int a = 0; a < NN; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i)
      sm.G[le][q][a][i] = (rr.dNf[q][a][0] * C[i][0] + rr.dNf[q][a][1] * C[i][1] + rr.dNf[q][a][2] * C[i][2]) * inv;
  const float wd = rr.wf[q] * det;
  sm.W[le][q] = wd;
  if constexpr (OP == FEA_OP_DIFFUSION) {
    const float x = f64_to_f32_rn(sm.X[le][0][0]) + xr;
    sm.S[le][q] = wd * (f64_to_f32_rn(P.k0) + f64_to_f32_rn(P.k2) * x * x);
  } else {
    sm.S[le][q] = wd;
  }
  return true;
}

template <int TYPE, int SLOT, int OP, int PREC, int SPLIT>
struct TileCfg {
  static constexpr int NN = nodes_of(TYPE);
  static constexpr int NQ = rule_nq(SLOT);
  static constexpr int D = OP == FEA_OP_DIFFUSION ? 1 : 3;
  static constexpr int LPE = NN * SPLIT;        // lanes per element
  static constexpr int EPW = 32 / LPE;          // elements per warp
  static constexpr int WARPS = 4;
  static constexpr int THREADS = 32 * WARPS;
  static constexpr int EPC = EPW * WARPS;       // elements per CTA
  static constexpr int NB = NN / SPLIT;         // columns per lane
  static constexpr bool kModal = TYPE == FEA_HEX8 && SLOT == kRuleHex8;
  static_assert(NN % SPLIT == 0, "SPLIT must divide the node count");
  static_assert(!kModal || (EPC * 8 % 32 == 0 && EPC * 8 <= THREADS), "modal hex geometry needs whole warps");
  using R = typename std::conditional<PREC == FEA_FP64, double, float>::type;
  using Smem = TileSmem<OP, PREC, NN, NQ, EPC>;
};

// phases 0 and 1 for the tile of elements [e0, e0 + EPC)
template <class Cfg, int OP, int PREC>
__device__ __forceinline__ void tile_geometry(typename Cfg::Smem& sm, const RefRule& rr, const AsmParams& P,
                                              int64_t e0, int64_t n_end) {
  constexpr int NN = Cfg::NN, NQ = Cfg::NQ, EPC = Cfg::EPC;
  constexpr bool kModal = Cfg::kModal;
  for (int t = threadIdx.x; t < EPC * NN; t += Cfg::THREADS) {
    const int le = t / NN, a = t % NN;
    const int64_t et = e0 + le;
    if (et < n_end) {
      const int64_t node = P.tconn[group_index(P, et) * NN + a];
      sm.X[le][a][0] = P.coords[3 * node + 0];
      sm.X[le][a][1] = P.coords[3 * node + 1];
      sm.X[le][a][2] = P.coords[3 * node + 2];
    }
  }
  if (threadIdx.x < EPC) sm.flag[threadIdx.x] = 0;
  __syncthreads();
  const bool all64 = PREC == FEA_FP64 || P.geo64;  // uniform over the grid
  if constexpr (kModal) {
    if (all64) {
      // trilinear hex in modal form: one lane per (element, corner p = point q);
      // EPC * 8 is a whole number of warps, so every lane of them takes part
      const int t = threadIdx.x;
      if (t < EPC * 8) {
        const int le = t >> 3, p = t & 7;
        const int64_t et = e0 + le;
        const bool valid = et < n_end;
        const int a = hex8_corner_node(p);
        double v[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) v[i] = valid ? sm.X[le][a][i] : 0.0;
        hex8_modal(v);
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 3; ++i) sm.X[le][p][i] = v[i];
        __syncwarp();
        double J[3][3];
        hex8_jacobian_pairs(sm.X[le], p, J);  // every lane: it exchanges columns with a partner lane
        if (valid) {
          double xq = 0.0;
          if constexpr (OP == FEA_OP_DIFFUSION) xq = hex8_modal_x(sm.X[le], p);
          geometry_finish<OP, NN>(sm, rr, le, p, original_id(P, et), J, 8.0, xq, P);
        }
      }
      __syncthreads();
      return;
    }
  }
  if constexpr (NN == 4) {  // tet4
    if (all64) {
      // a linear tet has one Jacobian (its shape-function derivatives are the
      // same at every point): J, its cofactors and det J once per element,
      // then each point's values from them
      for (int le = threadIdx.x; le < EPC; le += Cfg::THREADS) {
        const int64_t et = e0 + le;
        if (et >= n_end) continue;
        // with N = (1 - xi - eta - zeta, xi, eta, zeta) (ref_shape), dN_a/dxi_j
        // is 1 for a = j + 1 and 0 for the other nodes past node 0: column j
        // of J is the edge x_{j+1} - x_0, with no products
        double d[NN][3], J[3][3];
#pragma unroll
        for (int a = 1; a < NN; ++a)
#pragma unroll
          for (int i = 0; i < 3; ++i) d[a][i] = sm.X[le][a][i] - sm.X[le][0][i];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) J[i][j] = d[j + 1][i];
        double C[3][3];
        cofactors(J, C);
        const double det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
        if (!(det > 0.0)) latch_error(P.st, FEA_ERR_INVERTED_ELEMENT, (unsigned long long)original_id(P, et));
        if constexpr (PREC == FEA_FP64) {
#pragma unroll
          for (int q = 0; q < NQ; ++q) {
            double xq = sm.X[le][0][0];
#pragma unroll
            for (int a = 1; a < NN; ++a) xq += rr.N[q][a] * d[a][0];
            geometry_store<OP, NN>(sm, rr, le, q, C, det, 1.0, xq, P);
          }
        } else {
          // FP32 tiles: the FP32 roundings of C, det J and x at the points
          // replace the element's coordinates (read above), and the points'
          // values follow with one thread per point
          float xf[NQ];
#pragma unroll
          for (int q = 0; q < NQ; ++q) {
            double xq = sm.X[le][0][0];
#pragma unroll
            for (int a = 1; a < NN; ++a) xq += rr.N[q][a] * d[a][0];
            xf[q] = OP == FEA_OP_DIFFUSION ? f64_to_f32_rn(xq) : 0.0f;
          }
          float* o = reinterpret_cast<float*>(&sm.X[le][0][0]);
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) o[3 * i + j] = f64_to_f32_rn(C[i][j]);
          o[9] = f64_to_f32_rn(det);
#pragma unroll
          for (int q = 0; q < NQ; ++q) o[10 + q] = xf[q];
        }
      }
      if constexpr (PREC != FEA_FP64) {
        static_assert(10 + NQ <= NN * 3 * 2, "C, det J and x_q must fit the element's coordinate slot");
        __syncthreads();
        for (int t = threadIdx.x; t < EPC * NQ; t += Cfg::THREADS) {
          const int le = t / NQ, q = t % NQ;
          if (e0 + le >= n_end) continue;
          const float* o = reinterpret_cast<const float*>(&sm.X[le][0][0]);
          float Cf[3][3];
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) Cf[i][j] = o[3 * i + j];
          const float detf = o[9];
          const float inv = 1.0f / detf;
#pragma unroll
          for (int a = 0; a < NN; ++a)
#pragma unroll
            for (int i = 0; i < 3; ++i)
              sm.G[le][q][a][i] =
                  (rr.dNf[q][a][0] * Cf[i][0] + rr.dNf[q][a][1] * Cf[i][1] + rr.dNf[q][a][2] * Cf[i][2]) * inv;
          const float wdf = rr.wf[q] * detf;
          sm.W[le][q] = wdf;
          if constexpr (OP == FEA_OP_DIFFUSION) {
            const float x = o[10 + q];
            sm.S[le][q] = wdf * (f64_to_f32_rn(P.k0) + f64_to_f32_rn(P.k2) * x * x);
          } else {
            sm.S[le][q] = wdf;
          }
        }
      }
      __syncthreads();
      return;
    }
  }
  // FP64 hex (modal) and tet tiles have returned above
  if constexpr (!(PREC == FEA_FP64 && (kModal || NN == 4))) {
    if (all64) {
      // the differences to node 0 once per element, not once per point
      for (int t = threadIdx.x; t < EPC * (NN - 1) * 3; t += Cfg::THREADS) {
        const int le = t / ((NN - 1) * 3), r = t % ((NN - 1) * 3);
        if (e0 + le < n_end) sm.X[le][1 + r / 3][r % 3] -= sm.X[le][0][r % 3];
      }
      __syncthreads();
    }
    for (int t = threadIdx.x; t < EPC * NQ; t += Cfg::THREADS) {
      const int le = t / NQ, q = t % NQ;
      const int64_t et = e0 + le;
      if (et >= n_end) continue;
      if (all64) {
        geometry_fp64<OP, NN, true>(sm, rr, le, q, original_id(P, et), P);
      } else {
        if (!geometry_fp32<OP, NN>(sm, rr, le, q, P)) sm.flag[le] = 1;
      }
    }
    if (!all64) {
      __syncthreads();
      for (int t = threadIdx.x; t < EPC * NQ; t += Cfg::THREADS) {
        const int le = t / NQ, q = t % NQ;
        const int64_t et = e0 + le;
        if (et < n_end && sm.flag[le]) geometry_fp64<OP, NN>(sm, rr, le, q, original_id(P, et), P);
      }
    }
    __syncthreads();
  }
}

// phase 2: row block (a, columns b0 .. b0+NB) of element le, and its RHS
template <class Cfg, int OP>
__device__ __forceinline__ void row_block(const typename Cfg::Smem& sm, const RefRule& rr, const AsmParams& P,
                                          int le, int a, int b0, typename Cfg::R (&K)[Cfg::NB][Cfg::D][Cfg::D],
                                          typename Cfg::R (&rhs)[Cfg::D]) {
  using R = typename Cfg::R;
  constexpr int NB = Cfg::NB, D = Cfg::D, NQ = Cfg::NQ;
#pragma unroll
  for (int bb = 0; bb < NB; ++bb)
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
      for (int cc = 0; cc < D; ++cc) K[bb][c][cc] = R(0);
#pragma unroll
  for (int c = 0; c < D; ++c) rhs[c] = R(0);
  const R lam = (R)P.lam, mu = (R)P.mu;
#pragma unroll 1
  for (int q = 0; q < NQ; ++q) {
    const R s = sm.S[le][q];
    const R ga0 = sm.G[le][q][a][0], ga1 = sm.G[le][q][a][1], ga2 = sm.G[le][q][a][2];
    if constexpr (OP == FEA_OP_DIFFUSION) {
      const R sa0 = s * ga0, sa1 = s * ga1, sa2 = s * ga2;
#pragma unroll
      for (int bb = 0; bb < NB; ++bb) {
        const R* gb = sm.G[le][q][b0 + bb];
        K[bb][0][0] += sa0 * gb[0] + sa1 * gb[1] + sa2 * gb[2];
      }
    } else {
      const R gl[3] = {s * lam * ga0, s * lam * ga1, s * lam * ga2};
      const R gm[3] = {s * mu * ga0, s * mu * ga1, s * mu * ga2};
#pragma unroll
      for (int bb = 0; bb < NB; ++bb) {
        const R gb[3] = {sm.G[le][q][b0 + bb][0], sm.G[le][q][b0 + bb][1], sm.G[le][q][b0 + bb][2]};
        const R dot = gm[0] * gb[0] + gm[1] * gb[1] + gm[2] * gb[2];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int cc = 0; cc < 3; ++cc) K[bb][c][cc] += gl[c] * gb[cc] + gm[cc] * gb[c];
#pragma unroll
        for (int c = 0; c < 3; ++c) K[bb][c][c] += dot;
      }
    }
    if (b0 == 0) {
      R Nqa;
      if constexpr (std::is_same<R, double>::value)
        Nqa = rr.N[q][a];
      else
        Nqa = rr.Nf[q][a];
      const R wN = sm.W[le][q] * Nqa;
      if constexpr (OP == FEA_OP_DIFFUSION)
        rhs[0] += wN * (R)P.src;
      else
#pragma unroll
        for (int c = 0; c < 3; ++c) rhs[c] += wN * (R)P.f[c];
    }
  }
}

// Warp-cooperative reduction of FP32 elasticity row blocks.  A lane's row
// block holds, for each row c and column node b, three consecutive entries of
// A (24 bytes); one lane per entry scatters each warp-wide reduction over 32
// rows, while three neighbouring lanes on one 24-byte run and ten runs from
// one or two rows make each reduction touch about a third of the sectors
// (measured on GB300 with A in L2: 192 G reductions/s scattered, 443 G/s in
// runs of three).  The lanes hand their entries to the warp through the
// gradient table's shared memory, which row_block no longer needs: per warp
// the row starts (rbs), the column positions (ks, -1 for an idle lane) and PB
// columns' entries at a time (vals).
template <class Cfg, int SC>
struct CoopScatter {
  using Smem = typename Cfg::Smem;
  static constexpr int NB = Cfg::NB;
  static constexpr size_t kWarpBytes = sizeof(((Smem*)nullptr)->G) / Cfg::WARPS;
  static constexpr size_t kValsOff = 256 + 4 * 32 * NB;  // after rbs[32] and ks[32][NB]
  static constexpr int pb() {
    for (int p = NB; p > 0; --p)
      if (NB % p == 0 && kValsOff + 4 * 32 * 3 * p <= kWarpBytes) return p;
    return 0;
  }
  static constexpr int PB = pb();
  // hex8 with the 2x2x2 rule (PB = 4, 16-byte staging stores) is the tile it
  // serves; staged in pairs of columns, the tet4 items of the 256-mesh batch
  // made it slower (17.97 against 17.09 ms)
  static constexpr bool kOn = SC == FEA_SCATTER_ATOMIC && Cfg::D == 3 && Cfg::LPE == Cfg::NN && PB > 0 &&
                              std::is_same<typename Cfg::R, float>::value && kWarpBytes % 16 == 0 &&
                              (3 * PB) % 4 == 0;
};

// One tile of EPC elements starting at launch index e0 (elements at or past
// n_end are skipped): integrate, then scatter each row block (a, b0..b0+NB),
// warp-cooperatively when COOP is set.  Every thread of the CTA must call it;
// it ends with the shared memory free.
template <int TYPE, int SLOT, int OP, int PREC, int SPLIT, int SC, bool COOP = false>
__device__ __forceinline__ void tile_body(typename TileCfg<TYPE, SLOT, OP, PREC, SPLIT>::Smem& sm,
                                          const RefRule& rr, const AsmParams& P, int64_t e0, int64_t n_end) {
  using Cfg = TileCfg<TYPE, SLOT, OP, PREC, SPLIT>;
  using R = typename Cfg::R;
  constexpr int NN = Cfg::NN, D = Cfg::D, NB = Cfg::NB, LPE = Cfg::LPE, EPW = Cfg::EPW;
  tile_geometry<Cfg, OP, PREC>(sm, rr, P, e0, n_end);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int lw = lane / LPE;
  const int le = warp * EPW + lw;
  const int64_t et = e0 + le;
  if constexpr (COOP) {
    static_assert(CoopScatter<Cfg, SC>::kOn, "no cooperative scatter for this tile");
    using CS = CoopScatter<Cfg, SC>;
    constexpr int PB = CS::PB;
    static_assert(offsetof(typename Cfg::Smem, G) % 16 == 0, "staged entries need 16-byte rows");
    const bool active = lw < EPW && et < n_end;
    const int a = lane % LPE;
    R K[NB][D][D], rhs[D];
    int64_t rb[D] = {};
    int64_t node = 0;
    const int32_t* mp = nullptr;
    if (active) {
      row_block<Cfg, OP>(sm, rr, P, le, a, 0, K, rhs);
      const int64_t g = group_index(P, et);
      node = P.tconn[g * NN + a];
      const int64_t id = P.ids ? (int64_t)P.ids[g] : g;
      mp = P.node_map + (P.mapoff ? P.mapoff[g] : id * NN * NN) + a * NN;
#pragma unroll
      for (int c = 0; c < D; ++c) rb[c] = P.row_ptr[D * node + c];
    }
    __syncthreads();  // every row_block has read the gradient table
    unsigned char* wb = reinterpret_cast<unsigned char*>(&sm.G[0][0][0][0]) + warp * CS::kWarpBytes;
    int64_t* rbs = reinterpret_cast<int64_t*>(wb);
    int32_t* ks = reinterpret_cast<int32_t*>(wb + 256);
    float* vals = reinterpret_cast<float*>(wb + CS::kValsOff);
#pragma unroll
    for (int bb = 0; bb < NB; ++bb) ks[lane * NB + bb] = active ? mp[bb] : -1;
    // run j of a round: lanes 3j .. 3j+2 (lanes 30 and 31 rest)
    const int run = lane / 3, m = lane - 3 * run;
    constexpr int kRuns = 32 * PB, kRounds = (kRuns + 9) / 10;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      __syncwarp();
      rbs[lane] = rb[c];
#pragma unroll
      for (int part = 0; part < NB / PB; ++part) {
        __syncwarp();
        float4* v4 = reinterpret_cast<float4*>(vals + lane * PB * 3);
#pragma unroll
        for (int i = 0; i < 3 * PB / 4; ++i) {
          float t[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int f = 4 * i + u;
            t[u] = K[part * PB + f / 3][c][f % 3];
          }
          v4[i] = make_float4(t[0], t[1], t[2], t[3]);
        }
        __syncwarp();
#pragma unroll 2
        for (int r = 0; r < kRounds; ++r) {
          const int ch = 10 * r + run;  // run ch: lane ch / PB, column part * PB + ch % PB
          if (run < 10 && ch < kRuns) {
            const int s = ch / PB, j = ch - PB * s;
            const int32_t k = ks[s * NB + part * PB + j];
            if (k >= 0) red_add(P.A + rbs[s] + 3 * (int64_t)k + m, widen(vals[3 * ch + m]));
          }
        }
      }
    }
    if (active)
#pragma unroll
      for (int c = 0; c < D; ++c) red_add(P.b + D * node + c, widen(rhs[c]));
    __syncthreads();
    return;
  }
  if (lw < EPW && et < n_end) {
    const int r = lane % LPE;
    const int a = r % NN, b0 = (r / NN) * NB;

    R K[NB][D][D], rhs[D];
    row_block<Cfg, OP>(sm, rr, P, le, a, b0, K, rhs);

    const int64_t g = group_index(P, et);
    const int64_t node = P.tconn[g * NN + a];
    const int64_t id = P.ids ? (int64_t)P.ids[g] : g;
    const int64_t moff = P.mapoff ? P.mapoff[g] : id * NN * NN;
    const int32_t* mp = P.node_map + moff + a * NN + b0;
    int64_t rb[D];
#pragma unroll
    for (int c = 0; c < D; ++c) rb[c] = P.row_ptr[D * node + c];
    if constexpr (SC == FEA_SCATTER_MULTIDEP) {
      // this thread is the only writer of these entries (subdomain locks and
      // a local color class), but CTAs on other SMs wrote them before the
      // locks changed hands: read them from L2, a column's loads before its
      // stores (wider groups measured slower: registers)
#pragma unroll
      for (int bb = 0; bb < NB; ++bb) {
        const int64_t k = mp[bb];
        double old[D][D];
#pragma unroll
        for (int c = 0; c < D; ++c)
#pragma unroll
          for (int cc = 0; cc < D; ++cc) old[c][cc] = __ldcg(P.A + rb[c] + D * k + cc);
#pragma unroll
        for (int c = 0; c < D; ++c)
#pragma unroll
          for (int cc = 0; cc < D; ++cc) __stcg(P.A + rb[c] + D * k + cc, old[c][cc] + widen(K[bb][c][cc]));
      }
      if (b0 == 0) {
        double ob[D];
#pragma unroll
        for (int c = 0; c < D; ++c) ob[c] = __ldcg(P.b + D * node + c);
#pragma unroll
        for (int c = 0; c < D; ++c) __stcg(P.b + D * node + c, ob[c] + widen(rhs[c]));
      }
    } else {
#pragma unroll
      for (int bb = 0; bb < NB; ++bb) {
        const int64_t k = mp[bb];
#pragma unroll
        for (int c = 0; c < D; ++c)
#pragma unroll
          for (int cc = 0; cc < D; ++cc) scatter_add<SC>(P.A + rb[c] + D * k + cc, widen(K[bb][c][cc]));
      }
      if (b0 == 0)
#pragma unroll
        for (int c = 0; c < D; ++c) scatter_add<SC>(P.b + D * node + c, widen(rhs[c]));
    }
  }
  __syncthreads();
}

// Tile kernel: one tile per CTA.  Where the scatter is warp-cooperative its
// staging needs about 15 more registers than the plain one; at four CTAs per
// SM (128 registers) the hex8 elasticity FP32 atomic tile measured 5.69 ms
// per 128^3 step on GB300, against 6.83 at three CTAs and 6.20 with the
// plain scatter.  The other tiles keep the compiler's register choice (a
// bound of 0), and the persistent kernels the plain scatter: there the
// staging measured slower (8.22 against 7.48 ms; 256 meshes: 19.0 against
// 18.4 ms).
template <int TYPE, int SLOT, int OP, int PREC, int SPLIT, int SC>
__global__ void __launch_bounds__(128, CoopScatter<TileCfg<TYPE, SLOT, OP, PREC, SPLIT>, SC>::kOn ? 4 : 0)
    k_assemble_tile(const __grid_constant__ RefRule rr, const __grid_constant__ AsmParams P) {
  using Cfg = TileCfg<TYPE, SLOT, OP, PREC, SPLIT>;
  extern __shared__ __align__(16) unsigned char tile_smem[];
  auto& sm = *reinterpret_cast<typename Cfg::Smem*>(tile_smem);
  tile_body<TYPE, SLOT, OP, PREC, SPLIT, SC, CoopScatter<Cfg, SC>::kOn>(sm, rr, P, (int64_t)blockIdx.x * Cfg::EPC, P.n);
}

// ---------------------------------------------------------------------------
// persistent schedule: one launch over every element type (sched.cuh)
// ---------------------------------------------------------------------------
__constant__ RefRule c_rules[kNumRules];

struct PersistAsmArgs {
  AsmParams table[kNumTypes];  // entry t: the group of element type t
  int32_t slot[kNumTypes];     // its quadrature rule
  const AsmParams* tab;        // batches: device table of every (mesh, type) entry (overrides table)
  const int32_t* tab_slot;     // batches: rule slot per entry
  SchedArgs S;
};

template <int OP, int PREC>
struct PersistCfg {
  static constexpr int S2 = (OP == FEA_OP_ELASTICITY && PREC == FEA_FP64) ? 2 : 1;
  // CTAs per SM the any-type kernel is compiled for.  Its register count is
  // the largest tile body's plus the call sequence (120 for FP32 diffusion),
  // while the light types' own tiles need 46-56; measured on GB300 (4.53 M
  // mixed elements, FP32 diffusion: 4.26 ms with no bound, 4.00 at 5, 3.90 at
  // 6, 3.86 at 8; 256 elasticity meshes, FP32: 19.5 ms with no bound, 18.4
  // at 5, 19.9 at 6, where spills start to cost more than the occupancy
  // gains).  FP64 keeps the compiler's choice.  FP32 elasticity hex items
  // scatter warp-cooperatively (CoopScatter), which needs 4 CTAs per SM: the
  // 256 meshes 18.3 ms plain at 5, 19.3 cooperative at 5, 17.1 at 4, 18.8
  // at 3.  The hex-only kernel (ONLY) keeps the plain scatter: cooperative,
  // without a bound, it measured 8.56 against 7.46 ms on 2.1 M hexes.
  static constexpr int kMinBlocks = PREC == FEA_FP64 ? 1 : OP == FEA_OP_DIFFUSION ? 8 : 4;
  static constexpr bool kCoop = true;
  template <int TYPE, int SLOT, int SPLIT>
  static constexpr size_t bytes() { return sizeof(typename TileCfg<TYPE, SLOT, OP, PREC, SPLIT>::Smem); }
  static constexpr size_t mx(size_t a, size_t b) { return a > b ? a : b; }
  static constexpr size_t smem =
      mx(mx(mx(bytes<FEA_TET4, kRuleTet1, 1>(), bytes<FEA_TET4, kRuleTet4, 1>()), bytes<FEA_PYR5, kRulePyr8, 1>()),
         mx(bytes<FEA_PRISM6, kRulePrism6, S2>(), bytes<FEA_HEX8, kRuleHex8, S2>()));
};

template <int TYPE, int SLOT, int OP, int PREC, int SPLIT, int SC = FEA_SCATTER_ATOMIC, bool COOP = false>
__device__ __forceinline__ void persist_item(unsigned char* raw, const AsmParams& P, int64_t first, int64_t end) {
  using Cfg = TileCfg<TYPE, SLOT, OP, PREC, SPLIT>;
  auto& sm = *reinterpret_cast<typename Cfg::Smem*>(raw);
  constexpr bool kCoop = COOP && CoopScatter<Cfg, SC>::kOn;
  for (int64_t e0 = first; e0 < end; e0 += Cfg::EPC)
    tile_body<TYPE, SLOT, OP, PREC, SPLIT, SC, kCoop>(sm, c_rules[SLOT], P, e0, end);
}

// One item of the any-type kernel, not inlined: the switch over five inlined
// tile bodies made ptxas allocate well above the largest body's registers
// (FP32 diffusion: 128 against 72), which cut the all-type launch's
// occupancy; a call keeps the kernel near the largest body (96).
template <int TYPE, int SLOT, int OP, int PREC, int SPLIT>
__device__ __noinline__ void persist_item_call(unsigned char* raw, const AsmParams& P, int64_t first, int64_t end) {
  persist_item<TYPE, SLOT, OP, PREC, SPLIT, FEA_SCATTER_ATOMIC, PersistCfg<OP, PREC>::kCoop>(raw, P, first, end);
}

// ONLY >= 0: every item uses that rule slot (a single-type mesh), so the
// kernel holds one tile body and its register budget; -1: any element type
template <int OP, int PREC, int ONLY>
__global__ void __launch_bounds__(128, ONLY < 0 ? PersistCfg<OP, PREC>::kMinBlocks : 1)
    k_persistent(const __grid_constant__ PersistAsmArgs A) {
  constexpr int S2 = PersistCfg<OP, PREC>::S2;
  extern __shared__ __align__(16) unsigned char persist_smem[];
  __shared__ int s_item;
  sched_start(A.S);
  int k = 0;
  for (;;) {
    const int item = sched_next(A.S, k, &s_item);
    if (item < 0) break;
    const uint64_t t0 = global_ns();
    const WorkItem it = A.S.items[item];
    const int64_t first = it.first, end = (int64_t)it.first + it.count;
    // single mesh: entry t is type t, read at a constant offset of the
    // parameter space; batches: the device table
    if constexpr (ONLY == kRuleHex8) {
      persist_item<FEA_HEX8, kRuleHex8, OP, PREC, S2>(persist_smem, A.table[FEA_HEX8], first, end);
    } else if (A.tab) {
      const AsmParams& P = A.tab[it.entry];
      switch (A.tab_slot[it.entry]) {
        case kRuleTet1: persist_item_call<FEA_TET4, kRuleTet1, OP, PREC, 1>(persist_smem, P, first, end); break;
        case kRuleTet4: persist_item_call<FEA_TET4, kRuleTet4, OP, PREC, 1>(persist_smem, P, first, end); break;
        case kRulePyr8: persist_item_call<FEA_PYR5, kRulePyr8, OP, PREC, 1>(persist_smem, P, first, end); break;
        case kRulePrism6: persist_item_call<FEA_PRISM6, kRulePrism6, OP, PREC, S2>(persist_smem, P, first, end); break;
        default: persist_item_call<FEA_HEX8, kRuleHex8, OP, PREC, S2>(persist_smem, P, first, end); break;
      }
    } else {
      switch (A.slot[it.entry]) {
        case kRuleTet1: persist_item_call<FEA_TET4, kRuleTet1, OP, PREC, 1>(persist_smem, A.table[FEA_TET4], first, end); break;
        case kRuleTet4: persist_item_call<FEA_TET4, kRuleTet4, OP, PREC, 1>(persist_smem, A.table[FEA_TET4], first, end); break;
        case kRulePyr8: persist_item_call<FEA_PYR5, kRulePyr8, OP, PREC, 1>(persist_smem, A.table[FEA_PYR5], first, end); break;
        case kRulePrism6:
          persist_item_call<FEA_PRISM6, kRulePrism6, OP, PREC, S2>(persist_smem, A.table[FEA_PRISM6], first, end);
          break;
        default: persist_item_call<FEA_HEX8, kRuleHex8, OP, PREC, S2>(persist_smem, A.table[FEA_HEX8], first, end); break;
      }
    }
    sched_record(A.S, item, it.entry, t0);
  }
}

// ---------------------------------------------------------------------------
// commutative multidependences (FEA_SCATTER_MULTIDEP, Sec. 3.2.2): a CTA runs
// a subdomain only while it holds the lock of every subdomain of its
// neighbour list; the plan comes from multidep.cu
// ---------------------------------------------------------------------------
struct MdepArgs {
  AsmParams table[kNumTypes];  // entry t: the group of element type t, launch list = the plan's
  int32_t slot[kNumTypes];
  const WorkItem* items;       // subdomain k: elements first .. first + count of type entry
  const int64_t* nb_off;
  const int32_t* nb;           // neighbour lists, ascending, each with itself
  const int32_t* order;        // priority order
  const int64_t* cb_off;
  const int32_t* cb;           // color-class bounds (launch-list positions) per subdomain
  int32_t* state;              // 0 pending, 1 taken, 2 done
  int32_t* locks;              // 0 free
  int32_t* ctrl;               // [0] scan hint: no position before it is pending; [1] done count
  uint64_t* span;
  DevStatus* st;
  uint64_t timeout_ns;
  int32_t n_sub;
};

constexpr int kMdepWindows = 16;  // windows of 32 candidates one scan looks at

__device__ __forceinline__ int ld_relaxed(const int32_t* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// One lane: take subdomain k with every lock of its list (in ascending
// order), or give back what it took and hold nothing.
__device__ __forceinline__ bool mdep_try_take(const MdepArgs& A, int k) {
  if (atomicCAS(&A.state[k], 0, 1) != 0) return false;
  const int64_t j0 = A.nb_off[k], j1 = A.nb_off[k + 1];
  for (int64_t j = j0; j < j1; ++j) {
    if (atomicCAS(&A.locks[A.nb[j]], 0, 1) != 0) {
      for (int64_t i = j0; i < j; ++i) atomicExch(&A.locks[A.nb[i]], 0);
      atomicExch(&A.state[k], 0);
      return false;
    }
  }
  __threadfence();  // the locks are ours before any read of A
  return true;
}

// Warp 0 of the CTA: the next subdomain it runs, every lock of its list
// held (>= 0); -1 once every subdomain is done; -2 after searching in vain
// for longer than the timeout.  A scan walks the priority order in windows
// of 32 from the CTA's cursor (the hint when it starts over): lanes that see
// a pending subdomain whose locks all look free try to take it, lowest
// position first.  The hint moves over finished subdomains.
__device__ int mdep_next(const MdepArgs& A, int& cursor) {
  const int lane = threadIdx.x & 31;
  const uint64_t t0 = global_ns();
  for (;;) {
    if (ld_relaxed(&A.ctrl[1]) >= A.n_sub) return -1;
    const int h = ld_relaxed(&A.ctrl[0]);
    if (cursor < h || cursor >= A.n_sub) cursor = h;
    bool prefix = cursor == h;
    for (int w = 0; w < kMdepWindows && cursor < A.n_sub; ++w, cursor += 32) {
      const int pos = cursor + lane;
      int k = -1, st = 2;
      if (pos < A.n_sub) {
        k = A.order[pos];
        st = ld_relaxed(&A.state[k]);
      }
      const unsigned open = __ballot_sync(0xffffffffu, st != 2);
      if (prefix) {
        const int first = open ? cursor + __ffs(open) - 1 : (cursor + 32 < A.n_sub ? cursor + 32 : A.n_sub);
        if (lane == 0 && first > h) atomicMax(&A.ctrl[0], first);
        prefix = open == 0;
      }
      int busy = st != 0;
      if (!busy)
        for (int64_t j = A.nb_off[k]; j < A.nb_off[k + 1]; ++j) busy |= ld_relaxed(&A.locks[A.nb[j]]);
      unsigned m = __ballot_sync(0xffffffffu, !busy);
      while (m) {
        const int L = __ffs(m) - 1;
        m &= m - 1;
        int got = 0;
        if (lane == L) got = mdep_try_take(A, k);
        if (__shfl_sync(0xffffffffu, got, L)) return __shfl_sync(0xffffffffu, k, L);
      }
    }
    if (global_ns() - t0 > A.timeout_ns) return -2;
    __nanosleep(500);
  }
}

template <int OP, int PREC, int ONLY>
__global__ void __launch_bounds__(128) k_multidep(const __grid_constant__ MdepArgs A) {
  constexpr int S2 = PersistCfg<OP, PREC>::S2;
  constexpr int MD = FEA_SCATTER_MULTIDEP;
  extern __shared__ __align__(16) unsigned char mdep_smem[];
  __shared__ int s_sub;
  int cursor = 0;
  for (;;) {
    if (threadIdx.x < 32) {
      const int k = mdep_next(A, cursor);
      if (threadIdx.x == 0) {
        if (k == -2) latch_error(A.st, FEA_ERR_TIMEOUT, (unsigned long long)blockIdx.x);
        if (k >= 0 && A.span) A.span[2 * k] = global_ns();
        s_sub = k;
      }
    }
    __syncthreads();
    const int k = s_sub;
    if (k < 0) break;
    const WorkItem w = A.items[k];
    const AsmParams& P = A.table[w.entry];
    // the subdomain's local color classes, one after the other
    for (int64_t c = A.cb_off[k]; c + 1 < A.cb_off[k + 1]; ++c) {
      const int64_t p0 = A.cb[c], p1 = A.cb[c + 1];
      if constexpr (ONLY == kRuleHex8) {
        persist_item<FEA_HEX8, kRuleHex8, OP, PREC, S2, MD>(mdep_smem, P, p0, p1);
      } else {
        switch (A.slot[w.entry]) {
          case kRuleTet1: persist_item<FEA_TET4, kRuleTet1, OP, PREC, 1, MD>(mdep_smem, P, p0, p1); break;
          case kRuleTet4: persist_item<FEA_TET4, kRuleTet4, OP, PREC, 1, MD>(mdep_smem, P, p0, p1); break;
          case kRulePyr8: persist_item<FEA_PYR5, kRulePyr8, OP, PREC, 1, MD>(mdep_smem, P, p0, p1); break;
          case kRulePrism6: persist_item<FEA_PRISM6, kRulePrism6, OP, PREC, S2, MD>(mdep_smem, P, p0, p1); break;
          default: persist_item<FEA_HEX8, kRuleHex8, OP, PREC, S2, MD>(mdep_smem, P, p0, p1); break;
        }
      }
    }
    __syncthreads();  // every add of the subdomain is issued
    if (threadIdx.x == 0) {
      if (A.span) A.span[2 * k + 1] = global_ns();
      __threadfence();  // ... and visible before the locks change hands
      for (int64_t j = A.nb_off[k]; j < A.nb_off[k + 1]; ++j) atomicExch(&A.locks[A.nb[j]], 0);
      atomicExch(&A.state[k], 2);
      atomicAdd(&A.ctrl[1], 1);
    }
  }
}

int init_rule_constants() {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  FEA_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  if (dev < 64 && done[dev]) return FEA_OK;
  RefRule all[kNumRules];
  for (int r = 0; r < kNumRules; ++r) all[r] = host_rule(r);
  FEA_CUDA(cudaMemcpyToSymbol(c_rules, all, sizeof(all)));
  if (dev < 64) done[dev] = true;
  return init_rule_constants_j2();
}

static AsmParams base_params(const fea_operator* op, fea_mesh* m, const int64_t* row_ptr, const int32_t* node_map,
                             double* A, double* b) {
  AsmParams P;
  std::memset(&P, 0, sizeof(P));
  P.coords = m->coords;
  P.row_ptr = row_ptr;
  P.node_map = node_map;
  P.A = A;
  P.b = b;
  P.st = m->status;
  P.k0 = op->k0;
  P.k2 = op->k2;
  P.src = op->source;
  const double E = op->young, nu = op->poisson;
  P.lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  P.mu = E / (2.0 * (1.0 + nu));
  for (int c = 0; c < 3; ++c) P.f[c] = op->body_force[c];
  P.geo64 = op->precision != FEA_FP32_ADAPTIVE;
  return P;
}

static int rule_slot_of(int type, int tet_rule) {
  switch (type) {
    case FEA_TET4: return tet_rule ? kRuleTet4 : kRuleTet1;
    case FEA_PYR5: return kRulePyr8;
    case FEA_PRISM6: return kRulePrism6;
    default: return kRuleHex8;
  }
}

template <int OP, int PREC, int ONLY>
static int launch_persistent_k(const PersistAsmArgs& args, int n_ctas, bool dry, cudaStream_t s, int* grid_out) {
  constexpr size_t smem = ONLY == kRuleHex8 ? sizeof(typename TileCfg<FEA_HEX8, kRuleHex8, OP, PREC,
                                                                       PersistCfg<OP, PREC>::S2>::Smem)
                                            : PersistCfg<OP, PREC>::smem;
  auto kern = k_persistent<OP, PREC, ONLY>;
  if (smem > 48 * 1024) FEA_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int grid = n_ctas;
  if (grid <= 0) {
    int dev = 0, sms = 0, per_sm = 0;
    FEA_CUDA(cudaGetDevice(&dev));
    FEA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    FEA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, smem));
    grid = sms * (per_sm > 0 ? per_sm : 1);
  }
  if (grid_out) *grid_out = grid;
  if (!dry) {
    kern<<<grid, 128, smem, s>>>(args);
    FEA_CUDA(cudaGetLastError());
  }
  return FEA_OK;
}

// the hex-only kernel when every item is a 2x2x2 hex, else the generic one
template <int OP, int PREC>
static int launch_persistent_t(const PersistAsmArgs& args, int n_ctas, bool dry, cudaStream_t s, int* grid_out,
                               bool hex_only = false) {
  return hex_only ? launch_persistent_k<OP, PREC, kRuleHex8>(args, n_ctas, dry, s, grid_out)
                  : launch_persistent_k<OP, PREC, -1>(args, n_ctas, dry, s, grid_out);
}

// Persistent launch over a device table of (mesh, type) entries (batches).
int launch_persistent_batch(const fea_operator* op, const void* tab, const int32_t* tab_slot, const SchedArgs& S,
                            int n_ctas, bool dry, cudaStream_t s, int* grid_out) {
  PersistAsmArgs args;
  std::memset(&args, 0, sizeof(args));
  args.tab = static_cast<const AsmParams*>(tab);
  args.tab_slot = tab_slot;
  args.S = S;
  const bool f64 = op->precision == FEA_FP64;
  if (op->kind == FEA_OP_DIFFUSION)
    return f64 ? launch_persistent_t<FEA_OP_DIFFUSION, FEA_FP64>(args, n_ctas, dry, s, grid_out)
               : launch_persistent_t<FEA_OP_DIFFUSION, FEA_FP32_INTEGRATE>(args, n_ctas, dry, s, grid_out);
  return f64 ? launch_persistent_t<FEA_OP_ELASTICITY, FEA_FP64>(args, n_ctas, dry, s, grid_out)
             : launch_persistent_t<FEA_OP_ELASTICITY, FEA_FP32_INTEGRATE>(args, n_ctas, dry, s, grid_out);
}

// Size in bytes of one entry of the batch table, and the table entry of
// (mesh handle, type t) for the operator (host side, written into a buffer).
size_t batch_entry_bytes() { return sizeof(AsmParams); }

void batch_entry(const fea_operator* op, fea_mesh* m, int t, const int64_t* row_ptr, const int32_t* node_map,
                 double* A, double* b, void* out, int32_t* slot) {
  AsmParams P = base_params(op, m, row_ptr, node_map, A, b);
  const TypeGroup& g = m->group[t];
  P.tconn = g.conn;
  P.ids = g.ids;
  P.mapoff = g.mapoff;
  P.n = g.n;
  std::memcpy(out, &P, sizeof(P));
  *slot = rule_slot_of(t, op->tet_rule);
}

// Persistent launch of the diffusion / elasticity tile over every type group.
// n_ctas <= 0 selects the resident-CTA count (occupancy x SMs); the grid used
// is returned in *grid_out.  dry = true only computes the grid.
int launch_persistent_assemble(const fea_operator* op, fea_mesh* m, const int64_t* row_ptr, const int32_t* node_map,
                               double* A, double* b, const SchedArgs& S, int n_ctas, bool dry, cudaStream_t s,
                               int* grid_out) {
  PersistAsmArgs args;
  std::memset(&args, 0, sizeof(args));
  const AsmParams base = base_params(op, m, row_ptr, node_map, A, b);
  for (int t = 0; t < kNumTypes; ++t) {
    args.table[t] = base;
    const TypeGroup& g = m->group[t];
    args.table[t].tconn = g.conn;
    args.table[t].ids = g.ids;
    args.table[t].mapoff = g.mapoff;
    args.table[t].n = g.n;
    args.slot[t] = rule_slot_of(t, op->tet_rule);
  }
  args.S = S;
  // a mesh of hexes only runs the single-type kernel
  bool hex_only = m->group[FEA_HEX8].n > 0;
  for (int t = 0; t < kNumTypes; ++t)
    if (t != FEA_HEX8 && m->group[t].n) hex_only = false;
  int rc;
  const bool f64 = op->precision == FEA_FP64;
  if (op->kind == FEA_OP_DIFFUSION)
    rc = f64 ? launch_persistent_t<FEA_OP_DIFFUSION, FEA_FP64>(args, n_ctas, dry, s, grid_out, hex_only)
             : launch_persistent_t<FEA_OP_DIFFUSION, FEA_FP32_INTEGRATE>(args, n_ctas, dry, s, grid_out, hex_only);
  else
    rc = f64 ? launch_persistent_t<FEA_OP_ELASTICITY, FEA_FP64>(args, n_ctas, dry, s, grid_out, hex_only)
             : launch_persistent_t<FEA_OP_ELASTICITY, FEA_FP32_INTEGRATE>(args, n_ctas, dry, s, grid_out, hex_only);
  return rc;
}

template <int OP, int PREC, int ONLY>
static int launch_multidep_k(const MdepArgs& args, int n_ctas, cudaStream_t s) {
  constexpr size_t smem = ONLY == kRuleHex8 ? sizeof(typename TileCfg<FEA_HEX8, kRuleHex8, OP, PREC,
                                                                       PersistCfg<OP, PREC>::S2>::Smem)
                                            : PersistCfg<OP, PREC>::smem;
  auto kern = k_multidep<OP, PREC, ONLY>;
  if (smem > 48 * 1024) FEA_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int grid = n_ctas;
  if (grid <= 0) {
    int dev = 0, sms = 0, per_sm = 0;
    FEA_CUDA(cudaGetDevice(&dev));
    FEA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    FEA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, smem));
    grid = sms * (per_sm > 0 ? per_sm : 1);
  }
  if (grid > args.n_sub) grid = args.n_sub;
  kern<<<grid, 128, smem, s>>>(args);
  FEA_CUDA(cudaGetLastError());
  return FEA_OK;
}

// One persistent launch over the subdomains of the plan (A and b zeroed by
// the caller, the plan's state reset on the stream here).
int launch_multidep(const fea_operator* op, fea_mesh* m, const MultidepPlan& plan, const int64_t* row_ptr,
                    const int32_t* node_map, double* A, double* b, cudaStream_t s) {
  if (plan.n_sub == 0) return FEA_OK;
  int rc = init_rule_constants();
  if (rc) return rc;
  rc = reset_multidep(plan, s);
  if (rc) return rc;
  MdepArgs args;
  std::memset(&args, 0, sizeof(args));
  const AsmParams base = base_params(op, m, row_ptr, node_map, A, b);
  for (int t = 0; t < kNumTypes; ++t) {
    args.table[t] = base;
    const TypeGroup& g = m->group[t];
    args.table[t].tconn = g.conn;
    args.table[t].ids = g.ids;
    args.table[t].mapoff = g.mapoff;
    args.table[t].list = plan.lists[t];
    args.table[t].n = g.n;
    args.slot[t] = rule_slot_of(t, op->tet_rule);
  }
  args.items = plan.items;
  args.nb_off = plan.nb_off;
  args.nb = plan.nb;
  args.order = plan.order;
  args.cb_off = plan.cb_off;
  args.cb = plan.cb;
  args.state = plan.state;
  args.locks = plan.locks;
  args.ctrl = plan.ctrl;
  args.span = op->span_d;
  args.st = m->status;
  args.timeout_ns = 1000ull * (uint64_t)(op->lock_timeout_us > 0 ? op->lock_timeout_us : 1000000);
  args.n_sub = (int32_t)plan.n_sub;
  bool hex_only = m->group[FEA_HEX8].n > 0;
  for (int t = 0; t < kNumTypes; ++t)
    if (t != FEA_HEX8 && m->group[t].n) hex_only = false;
  const bool f64 = op->precision == FEA_FP64;
  if (op->kind == FEA_OP_DIFFUSION) {
    if (hex_only)
      return f64 ? launch_multidep_k<FEA_OP_DIFFUSION, FEA_FP64, kRuleHex8>(args, op->n_ctas, s)
                 : launch_multidep_k<FEA_OP_DIFFUSION, FEA_FP32_INTEGRATE, kRuleHex8>(args, op->n_ctas, s);
    return f64 ? launch_multidep_k<FEA_OP_DIFFUSION, FEA_FP64, -1>(args, op->n_ctas, s)
               : launch_multidep_k<FEA_OP_DIFFUSION, FEA_FP32_INTEGRATE, -1>(args, op->n_ctas, s);
  }
  if (hex_only)
    return f64 ? launch_multidep_k<FEA_OP_ELASTICITY, FEA_FP64, kRuleHex8>(args, op->n_ctas, s)
               : launch_multidep_k<FEA_OP_ELASTICITY, FEA_FP32_INTEGRATE, kRuleHex8>(args, op->n_ctas, s);
  return f64 ? launch_multidep_k<FEA_OP_ELASTICITY, FEA_FP64, -1>(args, op->n_ctas, s)
             : launch_multidep_k<FEA_OP_ELASTICITY, FEA_FP32_INTEGRATE, -1>(args, op->n_ctas, s);
}

// ---------------------------------------------------------------------------
// host dispatch
// ---------------------------------------------------------------------------
template <int TYPE, int SLOT, int OP, int PREC, int SPLIT, int SC>
static int launch_tile(const AsmParams& P, cudaStream_t s) {
  using Cfg = TileCfg<TYPE, SLOT, OP, PREC, SPLIT>;
  const unsigned grid = grid_for(P.n, Cfg::EPC);
  constexpr size_t smem = sizeof(typename Cfg::Smem);
  auto kern = k_assemble_tile<TYPE, SLOT, OP, PREC, SPLIT, SC>;
  if (smem > 48 * 1024) FEA_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<grid, Cfg::THREADS, smem, s>>>(host_rule(SLOT), P);
  FEA_CUDA(cudaGetLastError());
  return FEA_OK;
}

template <int OP, int PREC, int SC>
static int launch_group_sc(int type, int tet_rule, const AsmParams& P, cudaStream_t s) {
  // FP64 elasticity splits the columns of hex8 / prism6 over two lanes (register budget)
  constexpr int S2 = (OP == FEA_OP_ELASTICITY && PREC == FEA_FP64) ? 2 : 1;
  switch (type) {
    case FEA_TET4:
      return tet_rule ? launch_tile<FEA_TET4, kRuleTet4, OP, PREC, 1, SC>(P, s)
                      : launch_tile<FEA_TET4, kRuleTet1, OP, PREC, 1, SC>(P, s);
    case FEA_PYR5:
      return launch_tile<FEA_PYR5, kRulePyr8, OP, PREC, 1, SC>(P, s);
    case FEA_PRISM6:
      return launch_tile<FEA_PRISM6, kRulePrism6, OP, PREC, S2, SC>(P, s);
    default:
      return launch_tile<FEA_HEX8, kRuleHex8, OP, PREC, S2, SC>(P, s);
  }
}

template <int OP, int PREC>
static int launch_group(int type, int tet_rule, const AsmParams& P, cudaStream_t s) {
  return P.list ? launch_group_sc<OP, PREC, FEA_SCATTER_COLOR>(type, tet_rule, P, s)
                : launch_group_sc<OP, PREC, FEA_SCATTER_ATOMIC>(type, tet_rule, P, s);
}

int assemble(const fea_operator* op, fea_mesh* m, const int64_t* row_ptr, const int32_t* node_map, double* A,
             double* b, cudaStream_t s) {
  if (!op || !m || !row_ptr || !node_map || !A || !b) return fail(FEA_ERR_ARG, "fea_assemble: null argument");
  if (op->kind != FEA_OP_DIFFUSION && op->kind != FEA_OP_ELASTICITY && op->kind != FEA_OP_J2 &&
      op->kind != FEA_OP_NEOHOOKE)
    return fail(FEA_ERR_ARG, "fea_assemble: unknown operator kind");
  if (op->precision != FEA_FP64 && op->precision != FEA_FP32_INTEGRATE && op->precision != FEA_FP32_ADAPTIVE)
    return fail(FEA_ERR_ARG, "fea_assemble: unknown precision");
  if (op->scatter < FEA_SCATTER_ATOMIC || op->scatter > FEA_SCATTER_MULTIDEP)
    return fail(FEA_ERR_ARG, "fea_assemble: unknown scatter variant");
  if (op->tet_rule != 0 && op->tet_rule != 1) return fail(FEA_ERR_ARG, "fea_assemble: tet_rule must be 0 or 1");
  if (op->schedule < FEA_SCHED_PER_TYPE || op->schedule > FEA_SCHED_QUEUES_STEAL)
    return fail(FEA_ERR_ARG, "fea_assemble: unknown schedule");
  const int D = op->kind == FEA_OP_DIFFUSION ? 1 : 3;
  if (m->pattern_ndof != D || !m->pattern_built)
    return fail(FEA_ERR_ARG, "fea_assemble: build the pattern and map for ndof = " + std::to_string(D) + " first");
  if (op->scatter == FEA_SCATTER_MULTIDEP) {
    // its own persistent launch over the subdomains (the schedule is not used)
    if (op->kind == FEA_OP_J2 || op->kind == FEA_OP_NEOHOOKE)
      return fail(FEA_ERR_UNSUPPORTED, "fea_assemble: FEA_SCATTER_MULTIDEP assembles diffusion and elasticity");
    if (op->kind == FEA_OP_ELASTICITY && !(op->poisson > -1.0 && op->poisson < 0.5))
      return fail(FEA_ERR_ARG, "fea_assemble: poisson must be in (-1, 0.5)");
    if (op->chunk < 0 || op->n_ctas < 0 || op->lock_timeout_us < 0)
      return fail(FEA_ERR_ARG, "fea_assemble: chunk, n_ctas and lock_timeout_us must be >= 0");
    MultidepPlan* plan = nullptr;
    int rc = ensure_multidep_plan(m, op->chunk > 0 ? op->chunk : 128, &plan);  // host work on the first call only
    if (rc) return rc;
    cudaEvent_t* ev = (cudaEvent_t*)op->events;
    const int nev = ev ? op->n_events : 0;
    if (nev > 0) FEA_CUDA(cudaEventRecord(ev[0], s));
    FEA_CUDA(cudaMemsetAsync(A, 0, (int64_t)D * D * m->nnz_node * sizeof(double), s));
    FEA_CUDA(cudaMemsetAsync(b, 0, m->n_nodes * D * sizeof(double), s));
    if (nev > 1) FEA_CUDA(cudaEventRecord(ev[1], s));
    rc = launch_multidep(op, m, *plan, row_ptr, node_map, A, b, s);
    if (rc) return rc;
    for (int k = 2; k < nev; ++k) FEA_CUDA(cudaEventRecord(ev[k], s));
    return FEA_OK;
  }
  if (op->kind == FEA_OP_NEOHOOKE) return assemble_nh(op, m, row_ptr, node_map, A, b, s);
  if (op->schedule != FEA_SCHED_PER_TYPE) return assemble_persistent(op, m, row_ptr, node_map, A, b, s);
  if (op->kind == FEA_OP_J2) return assemble_j2(op, m, row_ptr, node_map, A, b, s);
  if (op->kind == FEA_OP_ELASTICITY) {
    if (!(op->poisson > -1.0 && op->poisson < 0.5)) return fail(FEA_ERR_ARG, "fea_assemble: poisson must be in (-1, 0.5)");
  }
  const int64_t nnz = (int64_t)D * D * m->nnz_node;
  cudaEvent_t* ev = (cudaEvent_t*)op->events;
  const int nev = ev ? op->n_events : 0;
  if (op->scatter == FEA_SCATTER_ROWS) {
    // every entry of A is written exactly once by its owner; only b rows of
    // nodes without elements would stay unwritten, so b alone is cleared
    RowsPlan* plan = nullptr;
    int prc = ensure_rows_plan(m, D, op->precision, s, &plan);  // host work on the first call only
    if (prc) return prc;
    if (nev > 0) FEA_CUDA(cudaEventRecord(ev[0], s));
    FEA_CUDA(cudaMemsetAsync(b, 0, m->n_nodes * D * sizeof(double), s));
    if (nev > 1) FEA_CUDA(cudaEventRecord(ev[1], s));
    void* records = nullptr;
    int geo = 0;
    int rc = geometry_pass(op, m, s, &records, &geo);
    if (rc) return rc;
    for (int k = 2; k < 2 + geo && k < nev; ++k) FEA_CUDA(cudaEventRecord(ev[k], s));
    rc = launch_task_kernel(op, *plan, records, row_ptr, A, b, m->status, s, nullptr);
    if (rc) return rc;
    for (int k = 2 + geo; k < nev; ++k) FEA_CUDA(cudaEventRecord(ev[k], s));
    return FEA_OK;
  }
  if (op->scatter == FEA_SCATTER_COLOR && !m->color) {
    int rc = build_color_plan(m, s);  // host-synchronous, first call only
    if (rc) return rc;
  }
  RowsPlan* bplan = nullptr;
  if (op->scatter == FEA_SCATTER_BLOCK) {
    int rc = ensure_blocks_plan(m, D, s, &bplan);  // host work on the first call only
    if (rc) return rc;
  }
  if (nev > 0) FEA_CUDA(cudaEventRecord(ev[0], s));
  if (bplan) {
    // the block-task kernels store every row whole except those of nodes on
    // block boundaries, which they add to: only those rows are cleared
    int rc = zero_block_rows(*bplan, row_ptr, A, s);
    if (rc) return rc;
  } else {
    FEA_CUDA(cudaMemsetAsync(A, 0, nnz * sizeof(double), s));
  }
  FEA_CUDA(cudaMemsetAsync(b, 0, m->n_nodes * D * sizeof(double), s));
  if (nev > 1) FEA_CUDA(cudaEventRecord(ev[1], s));
  if (op->scatter == FEA_SCATTER_BLOCK) {
    // geometry records (computed by the task kernel itself for hex meshes in
    // FP32-integrate), then one CTA per element block: interior entries are
    // stored, block-boundary entries added atomically into the zeroed A and b
    void* records = nullptr;
    int geo = 0;
    if (!fused_geometry(op, *bplan)) {
      int rc = geometry_pass(op, m, s, &records, &geo);
      if (rc) return rc;
    }
    for (int k = 2; k < 2 + geo && k < nev; ++k) FEA_CUDA(cudaEventRecord(ev[k], s));
    int rc = launch_task_kernel(op, *bplan, records, row_ptr, A, b, m->status, s, m);
    if (rc) return rc;
    for (int k = 2 + geo; k < nev; ++k) FEA_CUDA(cudaEventRecord(ev[k], s));
    return FEA_OK;
  }
  int launched = 0;

  AsmParams P;
  std::memset(&P, 0, sizeof(P));
  P.coords = m->coords;
  P.row_ptr = row_ptr;
  P.node_map = node_map;
  P.A = A;
  P.b = b;
  P.st = m->status;
  P.k0 = op->k0;
  P.k2 = op->k2;
  P.src = op->source;
  const double E = op->young, nu = op->poisson;
  P.lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  P.mu = E / (2.0 * (1.0 + nu));
  for (int c = 0; c < 3; ++c) P.f[c] = op->body_force[c];
  P.geo64 = op->precision != FEA_FP32_ADAPTIVE;
  auto run = [&](int t) -> int {
    int rc;
    if (op->kind == FEA_OP_DIFFUSION)
      rc = op->precision == FEA_FP64 ? launch_group<FEA_OP_DIFFUSION, FEA_FP64>(t, op->tet_rule, P, s)
                                     : launch_group<FEA_OP_DIFFUSION, FEA_FP32_INTEGRATE>(t, op->tet_rule, P, s);
    else
      rc = op->precision == FEA_FP64 ? launch_group<FEA_OP_ELASTICITY, FEA_FP64>(t, op->tet_rule, P, s)
                                     : launch_group<FEA_OP_ELASTICITY, FEA_FP32_INTEGRATE>(t, op->tet_rule, P, s);
    if (rc) return rc;
    if (2 + launched < nev) FEA_CUDA(cudaEventRecord(ev[2 + launched], s));
    ++launched;
    return FEA_OK;
  };
  if (op->scatter == FEA_SCATTER_COLOR) {
    // one launch per (color, element type): a launch never holds two elements
    // sharing a node, so its adds are plain read-modify-writes
    const ColorPlan& C = *m->color;
    for (int c = 0; c < C.n_colors; ++c)
      for (int t = 0; t < kNumTypes; ++t) {
        const size_t k = (size_t)c * kNumTypes + t;
        const int64_t n = C.seg_off[k + 1] - C.seg_off[k];
        if (!n) continue;
        const TypeGroup& g = m->group[t];
        P.tconn = g.conn;
        P.ids = g.ids;
        P.mapoff = g.mapoff;
        P.list = C.lists + C.seg_off[k];
        P.n = n;
        int rc = run(t);
        if (rc) return rc;
      }
    return FEA_OK;
  }
  for (int t = 0; t < kNumTypes; ++t) {
    const TypeGroup& g = m->group[t];
    if (!g.n) continue;
    P.tconn = g.conn;
    P.ids = g.ids;
    P.mapoff = g.mapoff;
    P.list = nullptr;
    P.n = g.n;
    int rc = run(t);
    if (rc) return rc;
  }
  return FEA_OK;
}

int assemble_launches(const fea_operator* op, const fea_mesh* m, int* n) {
  if (!op || !m || !n) return fail(FEA_ERR_ARG, "fea_assemble_launches: null argument");
  if (op->schedule != FEA_SCHED_PER_TYPE || op->scatter == FEA_SCATTER_MULTIDEP) {
    *n = 1;  // one persistent launch over every type (or every subdomain)
    return FEA_OK;
  }
  if (op->scatter == FEA_SCATTER_ROWS || op->scatter == FEA_SCATTER_BLOCK) {
    // geometry pass per element type, then the task kernel (block-task plans
    // of hex meshes in FP32-integrate compute the geometry in the task kernel)
    const bool fused = op->scatter == FEA_SCATTER_BLOCK && op->precision == FEA_FP32_INTEGRATE &&
                       m->group[FEA_HEX8].n == m->n_elems;
    *n = fused ? 1 : geometry_launches(m) + 1;
    // block-task plans clear the rows of A they add to first (one kernel,
    // unless the built plan has none: a mesh of one block)
    if (op->scatter == FEA_SCATTER_BLOCK && !(m->blocks && m->blocks->n_zero_runs == 0)) *n += 1;
    return FEA_OK;
  }
  if (op->scatter == FEA_SCATTER_COLOR) {
    if (!m->color) return fail(FEA_ERR_ARG, "fea_assemble_launches: the coloring is built by the first COLOR call");
    *n = color_launches(m);
    return FEA_OK;
  }
  int k = 0;
  for (int t = 0; t < kNumTypes; ++t) k += m->group[t].n > 0;
  *n = k;
  return FEA_OK;
}

}  // namespace fea
