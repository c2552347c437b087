// neohooke.cu -- Jacobian and internal force of the finite-strain solid
// (total Lagrangian, first Piola-Kirchhoff stress): the Newton step of the
// paper's structure solver, Sec. 2.2, whose costly part is the constitutive
// evaluation at every Gauss point (Sec. 5.2).
//
// The paper names no material; the engine reads it as the compressible
// neo-Hookean solid (Bonet and Wood 2008, Sec. 6.4.3):
//   Psi = mu/2 (F:F - 3) - mu ln J + lam/2 (ln J)^2,
//   P   = mu (F - F^-T) + lam ln J F^-T,
//   dP_iJ/dF_kL = mu d_ik d_JL + lam F^-1_Ji F^-1_Lk + (mu - lam ln J) F^-1_Jk F^-1_Li.
// Contracted with the reference gradients g_a = grad0 N_a, and with
// h_a = F^-T g_a (the spatial gradients), the element blocks are
//   A^e_ab = sum_q W_q [mu (g_a . g_b) I + lam h_a h_b^T + (mu - lam ln J) h_b h_a^T + m N_a N_b I],
//   f^e_a  = sum_q W_q P g_a,         W_q = w_q det J0_q,
// m N_a N_b I being the inertia term of the Newmark Jacobian.  Per Gauss
// point, FP64: the reference geometry, F = I + sum_a u_a (x) g_a, det F,
// F^-T, ln J and P.  The gradient products (h_a and the blocks) run in the
// tile precision (FP32 for FEA_FP32_INTEGRATE) and are added into A and b in
// FP64, by atomics (ATOMIC) or plain read-modify-writes (COLOR).
#include <cmath>
#include <cstring>
#include <type_traits>

#include "element.cuh"
#include "fea_internal.cuh"

namespace fea {

struct NHParams {
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
  double lam, mu, mass;
};

template <int TYPE, int SLOT, int PREC, int SPLIT>
struct NHCfg {
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
    R G[EPC][NQ][NN][3];  // g_a = grad0 N_a
    R H[EPC][NQ][NN][3];  // h_a = F^-T g_a
    R C[EPC][NQ][4];      // W mu, W lam, W (mu - lam ln J), W m
    R S[EPC][NQ][9];      // W P, row-major
  };
};

__device__ __forceinline__ int64_t nh_group_index(const NHParams& P, int64_t et) {
  return P.list ? (int64_t)P.list[et] : et;
}

// Phase 1 of point q of element le (FP64): J' = s J0 is the reference
// Jacobian scaled by a power of two s; writes the point's factors in the
// tile precision into shared memory.  MODAL (hex8, FP32 tiles): Ju' = s Ju
// is the displacement field's reference Jacobian from the modal transform of
// the nodal displacements, so F - I = Ju' C'^T / det' in FP64 and the
// reference gradients are formed in FP32 from C' and det' rounded once.
template <class Cfg, bool MODAL = false>
__device__ __forceinline__ void nh_point(typename Cfg::Smem& sm, const RefRule& rr, const NHParams& P, int le, int q,
                                         int64_t et, double (&J)[3][3], double s, const double (*Ju)[3] = nullptr) {
  using R = typename Cfg::R;
  constexpr int NN = Cfg::NN;
  const int64_t g = nh_group_index(P, et);
  const int64_t id = P.ids ? (int64_t)P.ids[g] : g;
  double C[3][3];
  cofactors(J, C);
  const double det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
  R gt[NN][3];  // g_a in the tile precision
  double F[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  double Fc[3][3], detF = 0.0;
  if (det > 0.0) {
    if constexpr (MODAL) {
      static_assert(!std::is_same<R, double>::value, "the modal path forms FP32 gradients");
      const double rdet = 1.0 / det;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) F[i][j] += (Ju[i][0] * C[j][0] + Ju[i][1] * C[j][1] + Ju[i][2] * C[j][2]) * rdet;
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
          for (int j = 0; j < 3; ++j) F[i][j] = fma(sm.U[le][a][i], gd[j], F[i][j]);
#pragma unroll
        for (int i = 0; i < 3; ++i) gt[a][i] = to_tile<R>(gd[i]);
      }
    }
    cofactors(F, Fc);  // cof F = det F * F^-T
    detF = F[0][0] * Fc[0][0] + F[0][1] * Fc[0][1] + F[0][2] * Fc[0][2];
  }
  if (!(det > 0.0) || !(detF > 0.0)) {
    // inverted in the reference configuration or by the deformation
    latch_error(P.st, FEA_ERR_INVERTED_ELEMENT, (unsigned long long)id);
#pragma unroll
    for (int k = 0; k < 4; ++k) sm.C[le][q][k] = R(0);
#pragma unroll
    for (int k = 0; k < 9; ++k) sm.S[le][q][k] = R(0);
#pragma unroll
    for (int a = 0; a < NN; ++a)
#pragma unroll
      for (int i = 0; i < 3; ++i) sm.G[le][q][a][i] = sm.H[le][q][a][i] = R(0);
    return;
  }
  const double rJ = 1.0 / detF;
  double Fit[3][3];  // F^-T
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Fit[i][j] = Fc[i][j] * rJ;
  const double lnJ = log(detF);
  const double W = rr.w[q] * det * (1.0 / (s * s * s));
  sm.C[le][q][0] = to_tile<R>(W * P.mu);
  sm.C[le][q][1] = to_tile<R>(W * P.lam);
  sm.C[le][q][2] = to_tile<R>(W * (P.mu - P.lam * lnJ));
  sm.C[le][q][3] = to_tile<R>(W * P.mass);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      sm.S[le][q][3 * i + j] = to_tile<R>(W * (P.mu * (F[i][j] - Fit[i][j]) + P.lam * lnJ * Fit[i][j]));
  // h_a = F^-T g_a in the tile precision, like the other gradient products
  R Ft[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Ft[i][j] = to_tile<R>(Fit[i][j]);
#pragma unroll
  for (int a = 0; a < NN; ++a) {
    const R g0 = gt[a][0], g1 = gt[a][1], g2 = gt[a][2];
    sm.G[le][q][a][0] = g0;
    sm.G[le][q][a][1] = g1;
    sm.G[le][q][a][2] = g2;
#pragma unroll
    for (int i = 0; i < 3; ++i) sm.H[le][q][a][i] = Ft[i][0] * g0 + Ft[i][1] * g1 + Ft[i][2] * g2;
  }
}

// One tile of EPC elements from launch index e0 (elements at or past n_end
// are skipped).  Every thread of the CTA calls it; it ends with a barrier.
template <int TYPE, int SLOT, int PREC, int SPLIT, int SC>
__device__ __forceinline__ void nh_tile_body(typename NHCfg<TYPE, SLOT, PREC, SPLIT>::Smem& sm, const RefRule& rr,
                                             const NHParams& P, int64_t e0, int64_t n_end) {
  using Cfg = NHCfg<TYPE, SLOT, PREC, SPLIT>;
  using R = typename Cfg::R;
  constexpr int NN = Cfg::NN, NQ = Cfg::NQ, EPC = Cfg::EPC, NB = Cfg::NB, LPE = Cfg::LPE, EPW = Cfg::EPW;
  // phase 0: coordinates and displacements of the tile's nodes
  for (int t = threadIdx.x; t < EPC * NN; t += Cfg::THREADS) {
    const int le = t / NN, a = t % NN;
    const int64_t et = e0 + le;
    if (et < n_end) {
      const int64_t node = P.tconn[nh_group_index(P, et) * NN + a];
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
      // FP32 tiles take the displacements to modal form as well (F then
      // needs no FP64 gradients); sm.U holds modal coefficients after
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
          nh_point<Cfg, true>(sm, rr, P, le, p, et, J, 8.0, Ju);
        else
          nh_point<Cfg>(sm, rr, P, le, p, et, J, 8.0);
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
      nh_point<Cfg>(sm, rr, P, le, q, et, J, 1.0);
    }
  }
  __syncthreads();

  // phase 2: lane (a, half) accumulates the row block (a, b0 .. b0 + NB)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int lw = lane / LPE;
  const int le = warp * EPW + lw;
  const int64_t et = e0 + le;
  if (lw < EPW && et < n_end) {
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
      const R wm = sm.C[le][q][0], wl = sm.C[le][q][1], wp = sm.C[le][q][2], wn = sm.C[le][q][3];
      const R ga[3] = {sm.G[le][q][a][0], sm.G[le][q][a][1], sm.G[le][q][a][2]};
      const R gm[3] = {wm * ga[0], wm * ga[1], wm * ga[2]};
      const R hl[3] = {wl * sm.H[le][q][a][0], wl * sm.H[le][q][a][1], wl * sm.H[le][q][a][2]};
      const R hp[3] = {wp * sm.H[le][q][a][0], wp * sm.H[le][q][a][1], wp * sm.H[le][q][a][2]};
      R Nqa;
      if constexpr (PREC == FEA_FP64)
        Nqa = rr.N[q][a];
      else
        Nqa = rr.Nf[q][a];
      const R mn = wn * Nqa;
#pragma unroll
      for (int bb = 0; bb < NB; ++bb) {
        const R gb[3] = {sm.G[le][q][b0 + bb][0], sm.G[le][q][b0 + bb][1], sm.G[le][q][b0 + bb][2]};
        const R hb[3] = {sm.H[le][q][b0 + bb][0], sm.H[le][q][b0 + bb][1], sm.H[le][q][b0 + bb][2]};
        R Nqb;
        if constexpr (PREC == FEA_FP64)
          Nqb = rr.N[q][b0 + bb];
        else
          Nqb = rr.Nf[q][b0 + bb];
        const R diag = gm[0] * gb[0] + gm[1] * gb[1] + gm[2] * gb[2] + mn * Nqb;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int cc = 0; cc < 3; ++cc) K[bb][c][cc] += hl[c] * hb[cc] + hb[c] * hp[cc];
#pragma unroll
        for (int c = 0; c < 3; ++c) K[bb][c][c] += diag;
      }
      if (b0 == 0) {
        const R* S = sm.S[le][q];
#pragma unroll
        for (int c = 0; c < 3; ++c) rhs[c] += S[3 * c] * ga[0] + S[3 * c + 1] * ga[1] + S[3 * c + 2] * ga[2];
      }
    }
    const int64_t g = nh_group_index(P, et);
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
__global__ void __launch_bounds__(128) k_nh_tile(const __grid_constant__ RefRule rr, const __grid_constant__ NHParams P) {
  using Cfg = NHCfg<TYPE, SLOT, PREC, SPLIT>;
  extern __shared__ __align__(16) unsigned char nh_smem_raw[];
  nh_tile_body<TYPE, SLOT, PREC, SPLIT, SC>(*reinterpret_cast<typename Cfg::Smem*>(nh_smem_raw), rr, P,
                                            (int64_t)blockIdx.x * Cfg::EPC, P.n);
}

template <int TYPE, int SLOT, int PREC, int SPLIT, int SC>
static int launch_nh(const NHParams& P, cudaStream_t s) {
  using Cfg = NHCfg<TYPE, SLOT, PREC, SPLIT>;
  constexpr size_t smem = sizeof(typename Cfg::Smem);
  static_assert(smem <= 227 * 1024, "finite-strain tile exceeds shared memory");
  auto kern = k_nh_tile<TYPE, SLOT, PREC, SPLIT, SC>;
  if (smem > 48 * 1024) FEA_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<grid_for(P.n, Cfg::EPC), Cfg::THREADS, smem, s>>>(host_rule(SLOT), P);
  FEA_CUDA(cudaGetLastError());
  return FEA_OK;
}

template <int PREC, int SC>
static int launch_nh_type(int type, const NHParams& P, cudaStream_t s) {
  constexpr int S2 = PREC == FEA_FP64 ? 2 : 1;  // FP64 splits the columns of hex8 / prism6 over two lanes
  switch (type) {
    case FEA_TET4: return launch_nh<FEA_TET4, kRuleTet4, PREC, 1, SC>(P, s);
    case FEA_PYR5: return launch_nh<FEA_PYR5, kRulePyr8, PREC, 1, SC>(P, s);
    case FEA_PRISM6: return launch_nh<FEA_PRISM6, kRulePrism6, PREC, S2, SC>(P, s);
    default: return launch_nh<FEA_HEX8, kRuleHex8, PREC, S2, SC>(P, s);
  }
}

int assemble_nh(const fea_operator* op, fea_mesh* m, const int64_t* row_ptr, const int32_t* node_map, double* A,
                double* b, cudaStream_t s) {
  if (op->scatter != FEA_SCATTER_ATOMIC && op->scatter != FEA_SCATTER_COLOR)
    return fail(FEA_ERR_UNSUPPORTED, "fea_assemble: the finite-strain solid supports the ATOMIC and COLOR scatters");
  if (op->schedule != FEA_SCHED_PER_TYPE)
    return fail(FEA_ERR_UNSUPPORTED, "fea_assemble: the finite-strain solid runs per element type");
  if (!op->u_d) return fail(FEA_ERR_ARG, "fea_assemble: the finite-strain solid needs the displacements u_d");
  if (!(op->poisson > -1.0 && op->poisson < 0.5)) return fail(FEA_ERR_ARG, "fea_assemble: poisson must be in (-1, 0.5)");
  if (!(op->mass >= 0.0)) return fail(FEA_ERR_ARG, "fea_assemble: mass must be >= 0");
  if (op->scatter == FEA_SCATTER_COLOR && !m->color) {
    int rc = build_color_plan(m, s);  // host-synchronous, first call only
    if (rc) return rc;
  }
  cudaEvent_t* ev = (cudaEvent_t*)op->events;
  const int nev = ev ? op->n_events : 0;
  if (nev > 0) FEA_CUDA(cudaEventRecord(ev[0], s));
  FEA_CUDA(cudaMemsetAsync(A, 0, 9 * m->nnz_node * sizeof(double), s));
  FEA_CUDA(cudaMemsetAsync(b, 0, m->n_nodes * 3 * sizeof(double), s));
  if (nev > 1) FEA_CUDA(cudaEventRecord(ev[1], s));

  NHParams P;
  std::memset(&P, 0, sizeof(P));
  P.coords = m->coords;
  P.row_ptr = row_ptr;
  P.node_map = node_map;
  P.A = A;
  P.b = b;
  P.st = m->status;
  P.u = op->u_d;
  const double E = op->young, nu = op->poisson;
  P.lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  P.mu = E / (2.0 * (1.0 + nu));
  P.mass = op->mass;
  const bool color = op->scatter == FEA_SCATTER_COLOR;
  int launched = 0;
  auto run = [&](int t) -> int {
    int rc;
    if (op->precision == FEA_FP64)
      rc = color ? launch_nh_type<FEA_FP64, FEA_SCATTER_COLOR>(t, P, s)
                 : launch_nh_type<FEA_FP64, FEA_SCATTER_ATOMIC>(t, P, s);
    else
      rc = color ? launch_nh_type<FEA_FP32_INTEGRATE, FEA_SCATTER_COLOR>(t, P, s)
                 : launch_nh_type<FEA_FP32_INTEGRATE, FEA_SCATTER_ATOMIC>(t, P, s);
    if (rc) return rc;
    if (2 + launched < nev) FEA_CUDA(cudaEventRecord(ev[2 + launched], s));
    ++launched;
    return FEA_OK;
  };
  if (color) {
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

}  // namespace fea
