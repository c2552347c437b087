// j2.cu -- tangent matrix and internal force of small-strain J2 plasticity
// with isotropic Voce hardening: the element loop of a nonlinear solid, whose
// Gauss-point constitutive update is the costly, data-dependent part (the
// paper's solid mechanics case, Sec. 2.2 and 5.2).
//
// Per Gauss point, in FP64: the strain eps = sym(grad u) of the nodal
// displacements, the radial return from the committed state (eps_p_n,
// alpha_n) with a scalar Newton iteration on the consistency condition
//   g(dg) = |s_tr| - 2 mu dg - sqrt(2/3) sigma_y(alpha_n + sqrt(2/3) dg) = 0,
//   sigma_y(a) = sigma0 + H a + (sigma_inf - sigma0)(1 - exp(-delta a)),
// and the consistent tangent
//   D_ep = kappa 1(x)1 + 2 mu theta I_dev - 2 mu theta_bar n(x)n
//        = lam' 1(x)1 + 2 mu' I_sym - beta n(x)n,
//   lam' = kappa - 2 mu theta / 3,  mu' = mu theta,  beta = 2 mu theta_bar,
//   theta = 1 - 2 mu dg / |s_tr|,  theta_bar = 1/(1 + sigma_y'/(3 mu)) - (1 - theta).
// The element blocks are then
//   A^e_ab = sum_q W_q [lam' g_a g_b^T + mu' g_b g_a^T + mu' (g_a . g_b) I - beta h_a h_b^T],
//   f^e_a  = sum_q W_q sigma g_a,       h_a = n g_a,  W_q = w_q det J_q,
// in the tile precision (FP32 for FEA_FP32_INTEGRATE: the return map and D_ep
// stay FP64, the D_ep B products are FP32; FP64 otherwise), accumulated into
// A and b in FP64 by atomics (ATOMIC) or plain read-modify-writes (COLOR).
#include <cmath>
#include <cstring>
#include <type_traits>

#include "element.cuh"
#include "fea_internal.cuh"
#include "sched.cuh"

namespace fea {

struct J2Params {
  const double* coords;
  const int32_t* tconn;   // [n][NN] packed connectivity of the type group
  const int32_t* ids;     // group index -> original id (nullptr: identity)
  const int64_t* mapoff;  // group index -> node_map offset (nullptr: id * NN^2)
  const int32_t* list;    // launch index -> group index (nullptr: identity; coloring)
  int64_t n;
  const int64_t* row_ptr;
  const int32_t* node_map;
  double* A;
  double* b;
  DevStatus* st;
  const double* u;
  const double* state_in;
  double* state_out;
  uint8_t* yield_out;
  uint8_t* iters_out;
  double* stress_out;     // element loop: [E][8][6] Cauchy stress per point slot (may be nullptr)
  double lam, mu, kappa;
  double s0, sinf, delta, hard, tol_g, tol_step;
  double mu2_3;           // 2 mu / 3: the factor 2 mu theta / 3 of an elastic point (theta = 1)
  int max_iter;
};

template <int TYPE, int SLOT, int PREC, int SPLIT>
struct J2Cfg {
  static constexpr int NN = nodes_of(TYPE);
  static constexpr int NQ = rule_nq(SLOT);
  static constexpr int LPE = NN * SPLIT;
  static constexpr int EPW = 32 / LPE;
  static constexpr int WARPS = 4;
  static constexpr int THREADS = 32 * WARPS;
  static constexpr int EPC = EPW * WARPS;
  static constexpr int NB = NN / SPLIT;
  static constexpr bool kModal = TYPE == FEA_HEX8 && SLOT == kRuleHex8;
  static_assert(NN % SPLIT == 0, "SPLIT must divide the node count");
  static_assert(!kModal || (EPC * 8 % 32 == 0 && EPC * 8 <= THREADS), "modal hex geometry needs whole warps");
  using R = typename std::conditional<PREC == FEA_FP64, double, float>::type;
  struct Smem {
    double X[EPC][NN][3];
    double U[EPC][NN][3];
    R G[EPC][NQ][NN][3];  // grad N_a
    R H[EPC][NQ][NN][3];  // h_a = n grad N_a
    R C[EPC][NQ][4];      // W, W lam', W mu', W beta
    R S[EPC][NQ][6];      // W sigma (xx, yy, zz, xy, yz, xz)
  };
};

__device__ __forceinline__ int64_t j2_group_index(const J2Params& P, int64_t et) {
  return P.list ? (int64_t)P.list[et] : et;
}

// Radial return at one point (all FP64).  eps, eps_p_n: tensor components.
struct J2Point {
  double sig[6], n[6], ep[6];
  double theta, theta_bar, alpha;
  int iters, yielded, ok;
};

__device__ __forceinline__ void j2_return(const J2Params& P, const double eps[6], const double epn[6], double an,
                                          J2Point& r) {
  const double r23 = 0.81649658092772603273;  // sqrt(2/3)
  double e[6], s[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) e[i] = eps[i] - epn[i];
  const double tr = e[0] + e[1] + e[2];
#pragma unroll
  for (int i = 0; i < 6; ++i) s[i] = 2.0 * P.mu * (e[i] - (i < 3 ? tr / 3.0 : 0.0));
  const double norm = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2] + 2.0 * (s[3] * s[3] + s[4] * s[4] + s[5] * s[5]));
  const double dsy = P.sinf - P.s0;
  // sigma_y(alpha_n); at alpha_n = 0 (a point that never yielded) it is s0
  // exactly, and the exp is not taken
  double sy_n = P.s0;
  if (an != 0.0) sy_n = P.s0 + P.hard * an + dsy * (1.0 - exp(-P.delta * an));
  r.theta = 1.0;
  r.theta_bar = 0.0;
  r.iters = 0;
  r.ok = 1;
#pragma unroll
  for (int i = 0; i < 6; ++i) r.n[i] = 0.0;
  if (norm - r23 * sy_n <= 0.0) {
#pragma unroll
    for (int i = 0; i < 6; ++i) r.ep[i] = epn[i];
    r.alpha = an;
    r.yielded = 0;
  } else {
    double dg = 0.0, ex = 1.0;
    int it = 0, ok = 0;
    bool ex_final = false;  // ex belongs to the final dg (no step after it)
    for (;;) {
      const double a = an + r23 * dg;
      ex = exp(-P.delta * a);
      const double g = norm - 2.0 * P.mu * dg - r23 * (P.s0 + P.hard * a + dsy * (1.0 - ex));
      if (fabs(g) <= P.tol_g * sy_n) {
        ok = 1;
        ex_final = true;
        break;
      }
      if (it == P.max_iter) {
        ex_final = true;
        break;
      }
      const double gp = -2.0 * P.mu - (2.0 / 3.0) * (P.hard + dsy * P.delta * ex);
      const double step = -g / gp;
      dg += step;
      ++it;
      if (fabs(step) <= P.tol_step) {
        ok = 1;
        break;
      }
    }
    r.iters = it;
    r.ok = ok;
    const double a = an + r23 * dg;
    // exp(-delta a) at the final dg: the loop's last value when it stopped at
    // the residual test or the iteration limit (the same a), else a new one
    const double slope = P.hard + dsy * P.delta * (ex_final ? ex : exp(-P.delta * a));
    const double inv = 1.0 / norm;
#pragma unroll
    for (int i = 0; i < 6; ++i) r.n[i] = s[i] * inv;
    r.theta = 1.0 - 2.0 * P.mu * dg * inv;
    r.theta_bar = 1.0 / (1.0 + slope / (3.0 * P.mu)) - (1.0 - r.theta);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      s[i] -= 2.0 * P.mu * dg * r.n[i];
      r.ep[i] = epn[i] + dg * r.n[i];
    }
    r.alpha = a;
    r.yielded = 1;
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) r.sig[i] = s[i] + (i < 3 ? P.kappa * tr : 0.0);
}

// Phase 1 of point q of element le: FP64 geometry, strain and return map;
// writes the per-point factors of the tile precision into shared memory.
// J' = s J is the reference Jacobian scaled by a power of two.  MODAL (hex8,
// FP32 tiles): Ju' = s Ju is the displacement field's reference Jacobian from
// the modal transform of the nodal displacements, and the displacement
// gradient is Ju J^-1 = Ju' C'^T / det' in FP64 (27 + 9 operations), so the
// shape-function gradients are only needed in the tile precision: formed in
// FP32 from C' and det' rounded once each, as the elasticity tile forms them.
template <class Cfg, bool MODAL = false>
__device__ __forceinline__ void j2_point(typename Cfg::Smem& sm, const RefRule& rr, const J2Params& P, int le, int q,
                                         int64_t et, double (&J)[3][3], double s, const double (*Ju)[3] = nullptr) {
  using R = typename Cfg::R;
  constexpr int NN = Cfg::NN;
  const int64_t g = j2_group_index(P, et);
  const int64_t id = P.ids ? (int64_t)P.ids[g] : g;
  double C[3][3];
  cofactors(J, C);
  const double det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
  if (!(det > 0.0)) {
    latch_error(P.st, FEA_ERR_INVERTED_ELEMENT, (unsigned long long)id);
#pragma unroll
    for (int k = 0; k < 4; ++k) sm.C[le][q][k] = R(0);
#pragma unroll
    for (int k = 0; k < 6; ++k) sm.S[le][q][k] = R(0);
#pragma unroll
    for (int a = 0; a < NN; ++a)
#pragma unroll
      for (int i = 0; i < 3; ++i) sm.G[le][q][a][i] = sm.H[le][q][a][i] = R(0);
    return;
  }
  // the displacement gradient H_ij = sum_a u_a,i g_a,j (FP64) and the
  // gradients g_a in the tile precision
  double Hu[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  R gt[NN][3];
  if constexpr (MODAL) {
    static_assert(!std::is_same<R, double>::value, "the modal strain path forms FP32 gradients");
    const double rdet = 1.0 / det;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) Hu[i][j] = (Ju[i][0] * C[j][0] + Ju[i][1] * C[j][1] + Ju[i][2] * C[j][2]) * rdet;
    float Cf[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) Cf[i][j] = f64_to_f32_rn(C[i][j]);
    const float invf = (float)s / f64_to_f32_rn(det);
#pragma unroll
    for (int a = 0; a < NN; ++a)
#pragma unroll
      for (int i = 0; i < 3; ++i)
        gt[a][i] = (rr.dNf[q][a][0] * Cf[i][0] + rr.dNf[q][a][1] * Cf[i][1] + rr.dNf[q][a][2] * Cf[i][2]) * invf;
  } else {
    const double inv = s / det;
#pragma unroll
    for (int a = 0; a < NN; ++a) {
      double gd[3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
        gd[i] = (rr.dN[q][a][0] * C[i][0] + rr.dN[q][a][1] * C[i][1] + rr.dN[q][a][2] * C[i][2]) * inv;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Hu[i][j] = fma(sm.U[le][a][i], gd[j], Hu[i][j]);
#pragma unroll
      for (int i = 0; i < 3; ++i) gt[a][i] = to_tile<R>(gd[i]);
    }
  }
  const double eps[6] = {Hu[0][0], Hu[1][1], Hu[2][2], 0.5 * (Hu[0][1] + Hu[1][0]), 0.5 * (Hu[1][2] + Hu[2][1]),
                         0.5 * (Hu[0][2] + Hu[2][0])};
  double epn[6] = {0, 0, 0, 0, 0, 0}, an = 0.0;
  const int64_t slot = id * 8 + q;
  if (P.state_in) {
    const double* sp = P.state_in + slot * 7;
#pragma unroll
    for (int i = 0; i < 6; ++i) epn[i] = sp[i];
    an = sp[6];
  }
  J2Point r;
  j2_return(P, eps, epn, an, r);
  if (!r.ok) latch_error(P.st, FEA_ERR_NO_CONVERGENCE, (unsigned long long)id);
  if (P.state_out) {
    double* sp = P.state_out + slot * 7;
#pragma unroll
    for (int i = 0; i < 6; ++i) sp[i] = r.ep[i];
    sp[6] = r.alpha;
  }
  if (P.yield_out) P.yield_out[slot] = (uint8_t)r.yielded;
  if (P.iters_out) P.iters_out[slot] = (uint8_t)r.iters;
  if (P.stress_out) {
#pragma unroll
    for (int i = 0; i < 6; ++i) P.stress_out[slot * 6 + i] = r.sig[i];
  }
  const double W = rr.w[q] * det * (1.0 / (s * s * s));
  sm.C[le][q][0] = to_tile<R>(W);
  // 2 mu theta / 3, from the host's 2 mu / 3 at an elastic point (the same
  // value: theta = 1 there), so that point takes no FP64 division
  const double mu2t_3 = r.yielded ? 2.0 * P.mu * r.theta / 3.0 : P.mu2_3;
  sm.C[le][q][1] = to_tile<R>(W * (P.kappa - mu2t_3));
  sm.C[le][q][2] = to_tile<R>(W * P.mu * r.theta);
  sm.C[le][q][3] = to_tile<R>(W * 2.0 * P.mu * r.theta_bar);
#pragma unroll
  for (int k = 0; k < 6; ++k) sm.S[le][q][k] = to_tile<R>(W * r.sig[k]);
  // h_a = n g_a in the tile precision (n = 0 at elastic points)
  const R n0 = to_tile<R>(r.n[0]), n1 = to_tile<R>(r.n[1]), n2 = to_tile<R>(r.n[2]), n3 = to_tile<R>(r.n[3]),
          n4 = to_tile<R>(r.n[4]), n5 = to_tile<R>(r.n[5]);
#pragma unroll
  for (int a = 0; a < NN; ++a) {
    const R g0 = gt[a][0], g1 = gt[a][1], g2 = gt[a][2];
    sm.G[le][q][a][0] = g0;
    sm.G[le][q][a][1] = g1;
    sm.G[le][q][a][2] = g2;
    sm.H[le][q][a][0] = n0 * g0 + n3 * g1 + n5 * g2;
    sm.H[le][q][a][1] = n3 * g0 + n1 * g1 + n4 * g2;
    sm.H[le][q][a][2] = n5 * g0 + n4 * g1 + n2 * g2;
  }
}

// One tile of EPC elements from launch index e0 (elements at or past n_end
// are skipped).  Every thread of the CTA calls it; it ends with a barrier.
// SCATTER = false is the element-wise loop: the Gauss-point update only.
template <int TYPE, int SLOT, int PREC, int SPLIT, int SC, bool SCATTER = true>
__device__ __forceinline__ void j2_tile_body(typename J2Cfg<TYPE, SLOT, PREC, SPLIT>::Smem& sm, const RefRule& rr,
                                             const J2Params& P, int64_t e0, int64_t n_end) {
  using Cfg = J2Cfg<TYPE, SLOT, PREC, SPLIT>;
  using R = typename Cfg::R;
  constexpr int NN = Cfg::NN, NQ = Cfg::NQ, EPC = Cfg::EPC, NB = Cfg::NB, LPE = Cfg::LPE, EPW = Cfg::EPW;
  // phase 0: coordinates and displacements of the tile's nodes
  for (int t = threadIdx.x; t < EPC * NN; t += Cfg::THREADS) {
    const int le = t / NN, a = t % NN;
    const int64_t et = e0 + le;
    if (et < n_end) {
      const int64_t node = P.tconn[j2_group_index(P, et) * NN + a];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        sm.X[le][a][i] = P.coords[3 * node + i];
        sm.U[le][a][i] = P.u[3 * node + i];
      }
    }
  }
  __syncthreads();
  // phase 1: one thread per (element, point)
  if constexpr (Cfg::kModal) {
    const int t = threadIdx.x;
    if (t < EPC * 8) {
      const int le = t >> 3, p = t & 7;
      const int64_t et = e0 + le;
      const bool valid = et < n_end;
      const int a = hex8_corner_node(p);
      // FP32 tiles take the displacements to modal form as well (the strain
      // then needs no FP64 gradients); sm.U holds modal coefficients after
      constexpr bool kModalU = PREC != FEA_FP64;
      double v[3], vu[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        v[i] = valid ? sm.X[le][a][i] : 0.0;
        vu[i] = valid ? sm.U[le][a][i] : 0.0;
      }
      hex8_modal(v);
      if constexpr (kModalU) hex8_modal(vu);
      __syncwarp();
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        sm.X[le][p][i] = v[i];
        if constexpr (kModalU) sm.U[le][p][i] = vu[i];
      }
      __syncwarp();
      // every lane forms its Jacobians (the lanes of an element exchange
      // columns); the valid ones use them
      double J[3][3], Ju[3][3];
      hex8_jacobian_pairs(sm.X[le], p, J);
      if constexpr (kModalU) hex8_jacobian_pairs(sm.U[le], p, Ju);
      if (valid) {
        if constexpr (kModalU)
          j2_point<Cfg, true>(sm, rr, P, le, p, et, J, 8.0, Ju);
        else
          j2_point<Cfg>(sm, rr, P, le, p, et, J, 8.0);
      }
    }
  } else {
    for (int t = threadIdx.x; t < EPC * NQ; t += Cfg::THREADS) {
      const int le = t / NQ, q = t % NQ;
      const int64_t et = e0 + le;
      if (et >= n_end) continue;
      double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
      for (int a = 1; a < NN; ++a) {
        const double d0 = sm.X[le][a][0] - sm.X[le][0][0];
        const double d1 = sm.X[le][a][1] - sm.X[le][0][1];
        const double d2 = sm.X[le][a][2] - sm.X[le][0][2];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          J[0][j] += d0 * rr.dN[q][a][j];
          J[1][j] += d1 * rr.dN[q][a][j];
          J[2][j] += d2 * rr.dN[q][a][j];
        }
      }
      j2_point<Cfg>(sm, rr, P, le, q, et, J, 1.0);
    }
  }
  __syncthreads();

  // phase 2: lane (a, half) accumulates the row block (a, b0 .. b0 + NB)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int lw = lane / LPE;
  const int le = warp * EPW + lw;
  const int64_t et = e0 + le;
  if (SCATTER && lw < EPW && et < n_end) {
    const int r = lane % LPE;
    const int a = r % NN, b0 = (r / NN) * NB;
    R K[NB][3][3], rhs[3] = {R(0), R(0), R(0)};
#pragma unroll
    for (int bb = 0; bb < NB; ++bb)
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) K[bb][c][cc] = R(0);
#pragma unroll 1
    for (int q = 0; q < NQ; ++q) {
      const R wl = sm.C[le][q][1], wm = sm.C[le][q][2], wb = sm.C[le][q][3];
      const R ga[3] = {sm.G[le][q][a][0], sm.G[le][q][a][1], sm.G[le][q][a][2]};
      const R gl[3] = {wl * ga[0], wl * ga[1], wl * ga[2]};
      const R gm[3] = {wm * ga[0], wm * ga[1], wm * ga[2]};
      const R hb[3] = {wb * sm.H[le][q][a][0], wb * sm.H[le][q][a][1], wb * sm.H[le][q][a][2]};
#pragma unroll
      for (int bb = 0; bb < NB; ++bb) {
        const R gb[3] = {sm.G[le][q][b0 + bb][0], sm.G[le][q][b0 + bb][1], sm.G[le][q][b0 + bb][2]};
        const R hh[3] = {sm.H[le][q][b0 + bb][0], sm.H[le][q][b0 + bb][1], sm.H[le][q][b0 + bb][2]};
        const R dot = gm[0] * gb[0] + gm[1] * gb[1] + gm[2] * gb[2];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int cc = 0; cc < 3; ++cc) K[bb][c][cc] += gl[c] * gb[cc] + gm[cc] * gb[c] - hb[c] * hh[cc];
#pragma unroll
        for (int c = 0; c < 3; ++c) K[bb][c][c] += dot;
      }
      if (b0 == 0) {
        const R* S = sm.S[le][q];
        rhs[0] += S[0] * ga[0] + S[3] * ga[1] + S[5] * ga[2];
        rhs[1] += S[3] * ga[0] + S[1] * ga[1] + S[4] * ga[2];
        rhs[2] += S[5] * ga[0] + S[4] * ga[1] + S[2] * ga[2];
      }
    }
    const int64_t g = j2_group_index(P, et);
    const int64_t node = P.tconn[g * NN + a];
    const int64_t id = P.ids ? (int64_t)P.ids[g] : g;
    const int64_t moff = P.mapoff ? P.mapoff[g] : id * NN * NN;
    const int32_t* mp = P.node_map + moff + a * NN + b0;
    int64_t rb[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) rb[c] = P.row_ptr[3 * node + c];
#pragma unroll
    for (int bb = 0; bb < NB; ++bb) {
      const int64_t k = mp[bb];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) scatter_add<SC>(P.A + rb[c] + 3 * k + cc, widen(K[bb][c][cc]));
    }
    if (b0 == 0)
#pragma unroll
      for (int c = 0; c < 3; ++c) scatter_add<SC>(P.b + 3 * node + c, widen(rhs[c]));
  }
  __syncthreads();
}

template <int TYPE, int SLOT, int PREC, int SPLIT, int SC>
__global__ void __launch_bounds__(128) k_j2_tile(const __grid_constant__ RefRule rr, const __grid_constant__ J2Params P) {
  using Cfg = J2Cfg<TYPE, SLOT, PREC, SPLIT>;
  extern __shared__ __align__(16) unsigned char j2_smem_raw[];
  j2_tile_body<TYPE, SLOT, PREC, SPLIT, SC>(*reinterpret_cast<typename Cfg::Smem*>(j2_smem_raw), rr, P,
                                            (int64_t)blockIdx.x * Cfg::EPC, P.n);
}

// element-wise loop: one tile of Gauss-point updates per CTA
template <int TYPE, int SLOT>
__global__ void __launch_bounds__(128) k_j2_points(const __grid_constant__ RefRule rr, const __grid_constant__ J2Params P) {
  using Cfg = J2Cfg<TYPE, SLOT, FEA_FP32_INTEGRATE, 1>;
  extern __shared__ __align__(16) unsigned char j2_smem_raw[];
  j2_tile_body<TYPE, SLOT, FEA_FP32_INTEGRATE, 1, FEA_SCATTER_ATOMIC, false>(
      *reinterpret_cast<typename Cfg::Smem*>(j2_smem_raw), rr, P, (int64_t)blockIdx.x * Cfg::EPC, P.n);
}

template <int TYPE, int SLOT>
static int launch_j2_points(const J2Params& P, cudaStream_t s) {
  using Cfg = J2Cfg<TYPE, SLOT, FEA_FP32_INTEGRATE, 1>;
  constexpr size_t smem = sizeof(typename Cfg::Smem);
  auto kern = k_j2_points<TYPE, SLOT>;
  if (smem > 48 * 1024) FEA_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<grid_for(P.n, Cfg::EPC), Cfg::THREADS, smem, s>>>(host_rule(SLOT), P);
  FEA_CUDA(cudaGetLastError());
  return FEA_OK;
}

template <int TYPE, int SLOT, int PREC, int SPLIT, int SC>
static int launch_j2(const J2Params& P, cudaStream_t s) {
  using Cfg = J2Cfg<TYPE, SLOT, PREC, SPLIT>;
  constexpr size_t smem = sizeof(typename Cfg::Smem);
  static_assert(smem <= 227 * 1024, "J2 tile exceeds shared memory");
  auto kern = k_j2_tile<TYPE, SLOT, PREC, SPLIT, SC>;
  if (smem > 48 * 1024) FEA_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const unsigned grid = grid_for(P.n, Cfg::EPC);
  kern<<<grid, Cfg::THREADS, smem, s>>>(host_rule(SLOT), P);
  FEA_CUDA(cudaGetLastError());
  return FEA_OK;
}

template <int PREC, int SC>
static int launch_j2_type(int type, const J2Params& P, cudaStream_t s) {
  constexpr int S2 = PREC == FEA_FP64 ? 2 : 1;  // FP64 splits the columns of hex8 / prism6 over two lanes
  switch (type) {
    case FEA_TET4: return launch_j2<FEA_TET4, kRuleTet4, PREC, 1, SC>(P, s);
    case FEA_PYR5: return launch_j2<FEA_PYR5, kRulePyr8, PREC, 1, SC>(P, s);
    case FEA_PRISM6: return launch_j2<FEA_PRISM6, kRulePrism6, PREC, S2, SC>(P, s);
    default: return launch_j2<FEA_HEX8, kRuleHex8, PREC, S2, SC>(P, s);
  }
}

static int launch_j2_any(int type, int precision, bool color, const J2Params& P, cudaStream_t s) {
  if (precision == FEA_FP64)
    return color ? launch_j2_type<FEA_FP64, FEA_SCATTER_COLOR>(type, P, s)
                 : launch_j2_type<FEA_FP64, FEA_SCATTER_ATOMIC>(type, P, s);
  return color ? launch_j2_type<FEA_FP32_INTEGRATE, FEA_SCATTER_COLOR>(type, P, s)
               : launch_j2_type<FEA_FP32_INTEGRATE, FEA_SCATTER_ATOMIC>(type, P, s);
}

// ---------------------------------------------------------------------------
// persistent schedule (sched.cuh): every element type in one launch
// ---------------------------------------------------------------------------
__constant__ RefRule c_rules_j2[kNumRules];

struct PersistJ2Args {
  J2Params table[kNumTypes];
  int32_t slot[kNumTypes];
  SchedArgs S;
};

template <int PREC>
struct PersistJ2Cfg {
  static constexpr int S2 = PREC == FEA_FP64 ? 2 : 1;
  template <int TYPE, int SLOT, int SPLIT>
  static constexpr size_t bytes() { return sizeof(typename J2Cfg<TYPE, SLOT, PREC, SPLIT>::Smem); }
  static constexpr size_t mx(size_t a, size_t b) { return a > b ? a : b; }
  static constexpr size_t smem = mx(mx(bytes<FEA_TET4, kRuleTet4, 1>(), bytes<FEA_PYR5, kRulePyr8, 1>()),
                                    mx(bytes<FEA_PRISM6, kRulePrism6, S2>(), bytes<FEA_HEX8, kRuleHex8, S2>()));
};

template <int TYPE, int SLOT, int PREC, int SPLIT, bool SCATTER>
__device__ __forceinline__ void persist_j2_item(unsigned char* raw, const J2Params& P, int64_t first, int64_t end) {
  using Cfg = J2Cfg<TYPE, SLOT, PREC, SPLIT>;
  auto& sm = *reinterpret_cast<typename Cfg::Smem*>(raw);
  for (int64_t e0 = first; e0 < end; e0 += Cfg::EPC)
    j2_tile_body<TYPE, SLOT, PREC, SPLIT, FEA_SCATTER_ATOMIC, SCATTER>(sm, c_rules_j2[SLOT], P, e0, end);
}

// ONLY == kRuleHex8: a mesh of hexes only (one tile body); -1: any type
template <int PREC, int ONLY, bool SCATTER>
__global__ void __launch_bounds__(128) k_persistent_j2(const __grid_constant__ PersistJ2Args A) {
  constexpr int S2 = PersistJ2Cfg<PREC>::S2;
  extern __shared__ __align__(16) unsigned char persist_j2_smem[];
  __shared__ int s_item;
  sched_start(A.S);
  int k = 0;
  for (;;) {
    const int item = sched_next(A.S, k, &s_item);
    if (item < 0) break;
    const uint64_t t0 = global_ns();
    const WorkItem it = A.S.items[item];
    const int64_t first = it.first, end = (int64_t)it.first + it.count;
    // entry t is type t: the parameters are read at constant offsets
    if constexpr (ONLY == kRuleHex8) {
      persist_j2_item<FEA_HEX8, kRuleHex8, PREC, S2, SCATTER>(persist_j2_smem, A.table[FEA_HEX8], first, end);
    } else {
      switch (A.slot[it.entry]) {
        case kRulePyr8: persist_j2_item<FEA_PYR5, kRulePyr8, PREC, 1, SCATTER>(persist_j2_smem, A.table[FEA_PYR5], first, end); break;
        case kRulePrism6:
          persist_j2_item<FEA_PRISM6, kRulePrism6, PREC, S2, SCATTER>(persist_j2_smem, A.table[FEA_PRISM6], first, end);
          break;
        case kRuleHex8: persist_j2_item<FEA_HEX8, kRuleHex8, PREC, S2, SCATTER>(persist_j2_smem, A.table[FEA_HEX8], first, end); break;
        default: persist_j2_item<FEA_TET4, kRuleTet4, PREC, 1, SCATTER>(persist_j2_smem, A.table[FEA_TET4], first, end); break;
      }
    }
    sched_record(A.S, item, it.entry, t0);
  }
}

int init_rule_constants_j2() {
  RefRule all[kNumRules];
  for (int r = 0; r < kNumRules; ++r) all[r] = host_rule(r);
  FEA_CUDA(cudaMemcpyToSymbol(c_rules_j2, all, sizeof(all)));
  return FEA_OK;
}

static int j2_validate(const fea_operator* op) {
  if (!op->u_d) return fail(FEA_ERR_ARG, "fea_assemble: J2 needs the displacements u_d");
  if (op->max_iter < 1 || op->max_iter > 255) return fail(FEA_ERR_ARG, "fea_assemble: J2 max_iter must be in [1, 255]");
  if (!(op->poisson > -1.0 && op->poisson < 0.5)) return fail(FEA_ERR_ARG, "fea_assemble: poisson must be in (-1, 0.5)");
  if (op->state_out_d && op->state_out_d == op->state_in_d)
    return fail(FEA_ERR_ARG, "fea_assemble: J2 state_out must not alias state_in");
  return FEA_OK;
}

static J2Params j2_base_params(const fea_operator* op, fea_mesh* m, const int64_t* row_ptr, const int32_t* node_map,
                               double* A, double* b) {
  J2Params P;
  std::memset(&P, 0, sizeof(P));
  P.coords = m->coords;
  P.row_ptr = row_ptr;
  P.node_map = node_map;
  P.A = A;
  P.b = b;
  P.st = m->status;
  P.u = op->u_d;
  P.state_in = op->state_in_d;
  P.state_out = op->state_out_d;
  P.yield_out = op->yield_out_d;
  P.iters_out = op->iters_out_d;
  const double E = op->young, nu = op->poisson;
  P.lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  P.mu = E / (2.0 * (1.0 + nu));
  P.kappa = P.lam + 2.0 * P.mu / 3.0;
  P.mu2_3 = 2.0 * P.mu / 3.0;
  P.s0 = op->sigma0;
  P.sinf = op->sigma_inf;
  P.delta = op->delta;
  P.hard = op->hardening;
  P.tol_g = op->tol_g;
  P.tol_step = op->tol_step;
  P.max_iter = op->max_iter;
  return P;
}

template <int PREC, int ONLY, bool SCATTER = true>
static int launch_persistent_j2_t(const PersistJ2Args& args, int n_ctas, bool dry, cudaStream_t s, int* grid_out) {
  constexpr size_t smem = ONLY == kRuleHex8
                              ? sizeof(typename J2Cfg<FEA_HEX8, kRuleHex8, PREC, PersistJ2Cfg<PREC>::S2>::Smem)
                              : PersistJ2Cfg<PREC>::smem;
  auto kern = k_persistent_j2<PREC, ONLY, SCATTER>;
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

int launch_persistent_j2(const fea_operator* op, fea_mesh* m, const int64_t* row_ptr, const int32_t* node_map,
                         double* A, double* b, const SchedArgs& S, int n_ctas, bool dry, cudaStream_t s,
                         int* grid_out, double* stress, bool points_only) {
  if (!dry) {
    int rc = j2_validate(op);
    if (rc) return rc;
  }
  PersistJ2Args args;
  std::memset(&args, 0, sizeof(args));
  J2Params base = j2_base_params(op, m, row_ptr, node_map, A, b);
  base.stress_out = stress;
  const int slots[kNumTypes] = {kRuleTet4, kRulePyr8, kRulePrism6, kRuleHex8};
  for (int t = 0; t < kNumTypes; ++t) {
    args.table[t] = base;
    const TypeGroup& g = m->group[t];
    args.table[t].tconn = g.conn;
    args.table[t].ids = g.ids;
    args.table[t].mapoff = g.mapoff;
    args.table[t].n = g.n;
    args.slot[t] = slots[t];
  }
  args.S = S;
  bool hex_only = m->group[FEA_HEX8].n > 0;
  for (int t = 0; t < kNumTypes; ++t)
    if (t != FEA_HEX8 && m->group[t].n) hex_only = false;
  if (points_only)  // the element-wise loop: Gauss-point updates only
    return hex_only ? launch_persistent_j2_t<FEA_FP32_INTEGRATE, kRuleHex8, false>(args, n_ctas, dry, s, grid_out)
                    : launch_persistent_j2_t<FEA_FP32_INTEGRATE, -1, false>(args, n_ctas, dry, s, grid_out);
  if (op->precision == FEA_FP64)
    return hex_only ? launch_persistent_j2_t<FEA_FP64, kRuleHex8>(args, n_ctas, dry, s, grid_out)
                    : launch_persistent_j2_t<FEA_FP64, -1>(args, n_ctas, dry, s, grid_out);
  return hex_only ? launch_persistent_j2_t<FEA_FP32_INTEGRATE, kRuleHex8>(args, n_ctas, dry, s, grid_out)
                  : launch_persistent_j2_t<FEA_FP32_INTEGRATE, -1>(args, n_ctas, dry, s, grid_out);
}

int assemble_j2(const fea_operator* op, fea_mesh* m, const int64_t* row_ptr, const int32_t* node_map, double* A,
                double* b, cudaStream_t s) {
  if (op->scatter != FEA_SCATTER_ATOMIC && op->scatter != FEA_SCATTER_COLOR)
    return fail(FEA_ERR_UNSUPPORTED, "fea_assemble: J2 supports the ATOMIC and COLOR scatters");
  int vrc = j2_validate(op);
  if (vrc) return vrc;
  if (op->scatter == FEA_SCATTER_COLOR && !m->color) {
    int rc = build_color_plan(m, s);
    if (rc) return rc;
  }
  cudaEvent_t* ev = (cudaEvent_t*)op->events;
  const int nev = ev ? op->n_events : 0;
  const int64_t nnz = 9 * m->nnz_node;
  if (nev > 0) FEA_CUDA(cudaEventRecord(ev[0], s));
  FEA_CUDA(cudaMemsetAsync(A, 0, nnz * sizeof(double), s));
  FEA_CUDA(cudaMemsetAsync(b, 0, m->n_nodes * 3 * sizeof(double), s));
  if (nev > 1) FEA_CUDA(cudaEventRecord(ev[1], s));

  J2Params P = j2_base_params(op, m, row_ptr, node_map, A, b);
  int launched = 0;
  auto run = [&](int t) -> int {
    int rc = launch_j2_any(t, op->precision, op->scatter == FEA_SCATTER_COLOR, P, s);
    if (rc) return rc;
    if (2 + launched < nev) FEA_CUDA(cudaEventRecord(ev[2 + launched], s));
    ++launched;
    return FEA_OK;
  };
  if (op->scatter == FEA_SCATTER_COLOR) {
    const ColorPlan& Cp = *m->color;
    for (int c = 0; c < Cp.n_colors; ++c)
      for (int t = 0; t < kNumTypes; ++t) {
        const size_t k = (size_t)c * kNumTypes + t;
        const int64_t n = Cp.seg_off[k + 1] - Cp.seg_off[k];
        if (!n) continue;
        const TypeGroup& g = m->group[t];
        P.tconn = g.conn;
        P.ids = g.ids;
        P.mapoff = g.mapoff;
        P.list = Cp.lists + Cp.seg_off[k];
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

// The element-wise loop (no scatter): the J2 update at every Gauss point,
// per type or by a persistent schedule (sched.cuh), writing the new state,
// the stress, the yield flags and the Newton iteration counts.
int element_loop_j2(const fea_operator* op, fea_mesh* m, double* stress, cudaStream_t s) {
  int rc = j2_validate(op);
  if (rc) return rc;
  if (op->schedule != FEA_SCHED_PER_TYPE) return element_loop_persistent(op, m, stress, s);
  cudaEvent_t* ev = (cudaEvent_t*)op->events;
  const int nev = ev ? op->n_events : 0;
  if (nev > 0) FEA_CUDA(cudaEventRecord(ev[0], s));
  if (nev > 1) FEA_CUDA(cudaEventRecord(ev[1], s));
  J2Params P = j2_base_params(op, m, nullptr, nullptr, nullptr, nullptr);
  P.stress_out = stress;
  int launched = 0;
  for (int t = 0; t < kNumTypes; ++t) {
    const TypeGroup& g = m->group[t];
    if (!g.n) continue;
    P.tconn = g.conn;
    P.ids = g.ids;
    P.mapoff = g.mapoff;
    P.list = nullptr;
    P.n = g.n;
    switch (t) {
      case FEA_TET4: rc = launch_j2_points<FEA_TET4, kRuleTet4>(P, s); break;
      case FEA_PYR5: rc = launch_j2_points<FEA_PYR5, kRulePyr8>(P, s); break;
      case FEA_PRISM6: rc = launch_j2_points<FEA_PRISM6, kRulePrism6>(P, s); break;
      default: rc = launch_j2_points<FEA_HEX8, kRuleHex8>(P, s); break;
    }
    if (rc) return rc;
    if (2 + launched < nev) FEA_CUDA(cudaEventRecord(ev[2 + launched], s));
    ++launched;
  }
  return FEA_OK;
}

}  // namespace fea

extern "C" int fea_element_loop(const fea_operator* op, fea_mesh* mesh, double* stress_d, void* stream) {
  using namespace fea;
  if (!op || !mesh) return fail(FEA_ERR_ARG, "fea_element_loop: null argument");
  if (op->kind != FEA_OP_J2) return fail(FEA_ERR_UNSUPPORTED, "fea_element_loop: the loop runs the J2 operator");
  if (op->schedule < FEA_SCHED_PER_TYPE || op->schedule > FEA_SCHED_QUEUES_STEAL)
    return fail(FEA_ERR_ARG, "fea_element_loop: unknown schedule");
  return element_loop_j2(op, mesh, stress_d, (cudaStream_t)stream);
}
