// geometry.cu -- the element geometry pass shared by the gather-style scatters.
//
// For every element and quadrature point q it evaluates the isoparametric map
// (J_ij = dx_i/dxi_j, det J, J^{-1}) and stores one record per element:
//   g^_a(q) = sqrt(w_q det J_q) J_q^{-T} grad_xi N_a(q)   [q][a][3]  (192 values)
//   W(q)    = w_q det J_q                                           (8 values)
//   K(q)    = k(x_q) = k0 + k2 x_q^2 (diffusion only)               (8 values)
// so that the contribution of one element to entry block (a, b) is
//   M = sum_q g^_a(q) (x) g^_b(q),   A^e_ab = lam M + mu M^T + mu tr(M) I   (elasticity)
//   A^e_ab = sum_q K(q) g^_a(q) . g^_b(q)                                  (diffusion)
// and its right-hand side b^e_a = sum_q W(q) N_a(q) f.
//
// FEA_FP32_INTEGRATE: J, its cofactors C and det J in FP64 for every element
// (the trilinear hex in modal form from its absolute corner coordinates, see
// hex8_modal -- the modal transform differences them exactly in FP64; other
// types from coordinates relative to node 0); C and det J are rounded to FP32
// once and the gradients formed from them in FP32.
// FEA_FP32_ADAPTIVE: coordinates relative to node 0 are subtracted in FP64 and
// rounded to FP32 once per (element, node); J, det J and J^{-1} are FP32 unless
// the element is distorted (Frobenius condition number of J above
// FEA_KAPPA_FP64 at some point, or a det J that FP32 cannot trust), in which
// case the element's geometry is redone in FP64 and rounded at the end.
// FEA_FP64: everything in FP64.  det J <= 0 latches FEA_ERR_INVERTED_ELEMENT.
#include <cmath>
#include <cstring>
#include <type_traits>

#include "element.cuh"
#include "fea_internal.cuh"
#include "geometry.cuh"

namespace fea {

struct GeoArgs {
  const double* coords;
  const int32_t* tconn;    // [n][NN] packed connectivity of the type group
  const int32_t* ids;      // [n] original element ids (nullptr: identity)
  int64_t n;
  void* rec;               // records indexed by original element id
  DevStatus* st;
  double k0, k2;
  int diffusion;
  int geo64;               // FP32 records: 1 = FP64 geometry for every element, 0 = adaptive
};

constexpr int kGeoThreads = 256;

// Record values of point q from the FP64 Jacobian J' = s J (s a power of two):
// det J = det'/s^3 and J^{-T} = s C'/det' with C' the cofactors of J'.
template <int NN, int PREC>
__device__ __forceinline__ void geo_finish(const RefRule& rr, const GeoArgs& P, int q, int64_t id, double (&J)[3][3],
                                           double s, double xq, void* recp) {
  double C[3][3];
  cofactors(J, C);
  const double det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
  if (!(det > 0.0)) {
    latch_error(P.st, FEA_ERR_INVERTED_ELEMENT, (unsigned long long)id);
    return;
  }
  if constexpr (PREC == FEA_FP64) {
    const double wd = rr.w[q] * det * (1.0 / (s * s * s));
    double* rec = static_cast<double*>(recp);
    const double sc = sqrt(wd) * s / det;
#pragma unroll
    for (int a = 0; a < NN; ++a)
#pragma unroll
      for (int i = 0; i < 3; ++i)
        rec[q * 24 + 3 * a + i] = (rr.dN[q][a][0] * C[i][0] + rr.dN[q][a][1] * C[i][1] + rr.dN[q][a][2] * C[i][2]) * sc;
    rec[kRecW + q] = wd;
    if (P.diffusion) rec[kRecK + q] = P.k0 + P.k2 * xq * xq;
  } else {
    // J^{-1} from the FP64 cofactors and determinant, rounded once each;
    // w det J follows in FP32 from the rounded determinant
    float* rec = static_cast<float*>(recp);
    float Cf[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) Cf[i][j] = f64_to_f32_rn(C[i][j]);
    const float detf = f64_to_f32_rn(det);
    const float wdf = rr.wf[q] * detf * (float)(1.0 / (s * s * s));
    const float sc = sqrtf(wdf) * (float)s / detf;
#pragma unroll
    for (int a = 0; a < NN; ++a)
#pragma unroll
      for (int i = 0; i < 3; ++i)
        rec[q * 24 + 3 * a + i] =
            (rr.dNf[q][a][0] * Cf[i][0] + rr.dNf[q][a][1] * Cf[i][1] + rr.dNf[q][a][2] * Cf[i][2]) * sc;
    rec[kRecW + q] = wdf;
    if (P.diffusion) {
      const float x = f64_to_f32_rn(xq);
      rec[kRecK + q] = f64_to_f32_rn(P.k0) + f64_to_f32_rn(P.k2) * x * x;
    }
  }
}

template <int TYPE, int SLOT, int PREC>
__global__ void __launch_bounds__(kGeoThreads) k_geometry(const __grid_constant__ RefRule rr,
                                                          const __grid_constant__ GeoArgs P) {
  using R = typename std::conditional<PREC == FEA_FP64, double, float>::type;
  constexpr int NN = nodes_of(TYPE);
  constexpr int NQ = rule_nq(SLOT);
  constexpr int EPC = kGeoThreads / 8;  // elements per CTA (8 threads each)
  constexpr bool kModal = TYPE == FEA_HEX8 && SLOT == kRuleHex8;
  __shared__ double sX[EPC][8][3];      // node coordinates (modal hex: then the c_k)
  __shared__ float sD[EPC][8][3];
  __shared__ int sFlag[EPC];
  const int le = threadIdx.x >> 3, lane8 = threadIdx.x & 7;
  const int64_t et = (int64_t)blockIdx.x * EPC + le;
  const bool valid = et < P.n;
  const int64_t id = valid ? (P.ids ? (int64_t)P.ids[et] : et) : 0;
  // node coordinates: thread (le, a) loads node a
  if (valid && lane8 < NN) {
    const int64_t node = P.tconn[et * NN + lane8];
    sX[le][lane8][0] = P.coords[3 * node + 0];
    sX[le][lane8][1] = P.coords[3 * node + 1];
    sX[le][lane8][2] = P.coords[3 * node + 2];
  }
  if (lane8 == 0) sFlag[le] = 0;
  __syncthreads();
  R* rec = reinterpret_cast<R*>(P.rec) + id * kRecStride;
  const int q = lane8;
  const bool all64 = PREC == FEA_FP64 || P.geo64;  // uniform over the grid
  if (!all64) {
    // adaptive: FP32 geometry on coordinates relative to node 0, distorted
    // elements flagged for the FP64 redo below
    if (valid && lane8 < NN) {
      sD[le][lane8][0] = f64_to_f32_rn(sX[le][lane8][0] - sX[le][0][0]);
      sD[le][lane8][1] = f64_to_f32_rn(sX[le][lane8][1] - sX[le][0][1]);
      sD[le][lane8][2] = f64_to_f32_rn(sX[le][lane8][2] - sX[le][0][2]);
    }
    __syncthreads();
    if (valid && q < NQ) {
      float J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
      float xr = 0.0f;
#pragma unroll
      for (int a = 1; a < NN; ++a) {
        const float d0 = sD[le][a][0], d1 = sD[le][a][1], d2 = sD[le][a][2];
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
      const float kappa2_max = (float)(FEA_KAPPA_FP64 * FEA_KAPPA_FP64);
      if (!(det > 0.0f) || !(nj * nc <= kappa2_max * det * det)) {
        sFlag[le] = 1;
      } else {
        const float wd = rr.wf[q] * det;
        const float sc = sqrtf(wd) / det;
#pragma unroll
        for (int a = 0; a < NN; ++a)
#pragma unroll
          for (int i = 0; i < 3; ++i)
            rec[q * 24 + 3 * a + i] =
                (R)((rr.dNf[q][a][0] * C[i][0] + rr.dNf[q][a][1] * C[i][1] + rr.dNf[q][a][2] * C[i][2]) * sc);
        rec[kRecW + q] = (R)wd;
        if (P.diffusion) {
          const float x = f64_to_f32_rn(sX[le][0][0]) + xr;
          rec[kRecK + q] = (R)(f64_to_f32_rn(P.k0) + f64_to_f32_rn(P.k2) * x * x);
        }
      }
    }
    __syncthreads();
  }
  if constexpr (kModal) {
    if (all64) {
      // every lane of the warp takes part in the butterfly (tail lanes on zeros)
      const int p = lane8;
      const int a = hex8_corner_node(p);
      double v[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) v[i] = valid ? sX[le][a][i] : 0.0;
      hex8_modal(v);
      __syncwarp();
#pragma unroll
      for (int i = 0; i < 3; ++i) sX[le][p][i] = v[i];
      __syncwarp();
      double J[3][3];
      hex8_jacobian_pairs(sX[le], q, J);  // every lane: it exchanges columns with a partner lane
      if (valid) {
        double xq = 0.0;
        if (P.diffusion) xq = hex8_modal_x(sX[le], q);
        geo_finish<NN, PREC>(rr, P, q, id, J, 8.0, xq, rec);
      }
      return;
    }
  }
  const bool need64 = valid && q < NQ && (all64 || sFlag[le]);
  if (need64) {
    double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    double xq = sX[le][0][0];
#pragma unroll
    for (int a = 1; a < NN; ++a) {
      const double d0 = sX[le][a][0] - sX[le][0][0];
      const double d1 = sX[le][a][1] - sX[le][0][1];
      const double d2 = sX[le][a][2] - sX[le][0][2];
      xq += rr.N[q][a] * d0;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        J[0][j] += d0 * rr.dN[q][a][j];
        J[1][j] += d1 * rr.dN[q][a][j];
        J[2][j] += d2 * rr.dN[q][a][j];
      }
    }
    geo_finish<NN, PREC>(rr, P, q, id, J, 1.0, xq, rec);
  }
}

template <int TYPE, int SLOT, int PREC>
static int launch_geo(const GeoArgs& P, cudaStream_t s) {
  const unsigned grid = grid_for(P.n, kGeoThreads / 8);
  k_geometry<TYPE, SLOT, PREC><<<grid, kGeoThreads, 0, s>>>(host_rule(SLOT), P);
  FEA_CUDA(cudaGetLastError());
  return FEA_OK;
}

template <int PREC>
static int launch_geo_type(int type, int tet_rule, const GeoArgs& P, cudaStream_t s) {
  switch (type) {
    case FEA_TET4:
      return tet_rule ? launch_geo<FEA_TET4, kRuleTet4, PREC>(P, s) : launch_geo<FEA_TET4, kRuleTet1, PREC>(P, s);
    case FEA_PYR5: return launch_geo<FEA_PYR5, kRulePyr8, PREC>(P, s);
    case FEA_PRISM6: return launch_geo<FEA_PRISM6, kRulePrism6, PREC>(P, s);
    default: return launch_geo<FEA_HEX8, kRuleHex8, PREC>(P, s);
  }
}

int geometry_pass(const fea_operator* op, fea_mesh* m, cudaStream_t s, void** records, int* launched) {
  const int pi = op->precision == FEA_FP64 ? 0 : 1;
  const size_t rb = (op->precision == FEA_FP64 ? 8 : 4) * (size_t)kRecStride * (size_t)m->n_elems;
  if (!m->geo[pi]) {
    cudaError_t e = cudaMalloc(&m->geo[pi], rb);
    if (e != cudaSuccess) {
      m->geo[pi] = nullptr;
      return fail(FEA_ERR_OOM, "geometry records: cudaMalloc of " + std::to_string(rb) + " bytes failed");
    }
  }
  GeoArgs P;
  std::memset(&P, 0, sizeof(P));
  P.coords = m->coords;
  P.rec = m->geo[pi];
  P.st = m->status;
  P.k0 = op->k0;
  P.k2 = op->k2;
  P.diffusion = op->kind == FEA_OP_DIFFUSION;
  P.geo64 = op->precision != FEA_FP32_ADAPTIVE;
  int k = 0;
  for (int t = 0; t < kNumTypes; ++t) {
    const TypeGroup& g = m->group[t];
    if (!g.n) continue;
    P.tconn = g.conn;
    P.ids = g.ids;
    P.n = g.n;
    const int rc = op->precision == FEA_FP64 ? launch_geo_type<FEA_FP64>(t, op->tet_rule, P, s)
                                             : launch_geo_type<FEA_FP32_INTEGRATE>(t, op->tet_rule, P, s);
    if (rc) return rc;
    ++k;
  }
  *records = m->geo[pi];
  if (launched) *launched = k;
  return FEA_OK;
}

int geometry_launches(const fea_mesh* m) {
  int k = 0;
  for (int t = 0; t < kNumTypes; ++t) k += m->group[t].n > 0;
  return k;
}

}  // namespace fea
