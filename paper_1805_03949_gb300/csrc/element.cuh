// element.cuh -- reference elements, quadrature rules and the per-quadrature
// point geometry shared by every assembly kernel of the engine.
//
// Element formulations (the paper states the PDEs, Sec. 2.1.1 and 2.2.1, but
// no element formulation; these are the textbook Galerkin ones):
//   diffusion  A^e_ab = sum_q w_q detJ_q k(x_q) grad N_a . grad N_b,
//              b^e_a  = sum_q w_q detJ_q f N_a,            k(x) = k0 + k2 x^2
//   elasticity A^e_(a,c)(b,c') = sum_q w_q detJ_q [lam g_a,c g_b,c' +
//              mu g_a,c' g_b,c + mu delta_cc' g_a . g_b]  (= B_a^T D B_b for
//              isotropic D), b^e_(a,c) = sum_q w_q detJ_q f_c N_a
// with g_a = grad N_a = J^{-T} grad_xi N_a and J_ij = dx_i / dxi_j.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fea_internal.cuh"

namespace fea {

// quadrature rule slots
enum RuleSlot { kRuleTet1 = 0, kRuleTet4 = 1, kRulePyr8 = 2, kRulePrism6 = 3, kRuleHex8 = 4, kNumRules = 5 };

__host__ __device__ constexpr int rule_nq(int slot) {
  return slot == kRuleTet1 ? 1 : slot == kRuleTet4 ? 4 : slot == kRulePrism6 ? 6 : 8;
}
__host__ __device__ constexpr int rule_type(int slot) {
  return slot <= kRuleTet4 ? FEA_TET4 : slot == kRulePyr8 ? FEA_PYR5 : slot == kRulePrism6 ? FEA_PRISM6 : FEA_HEX8;
}

// Reference values at the quadrature points of one rule.
struct RefRule {
  double w[8];
  double N[8][8];       // [q][a]
  double dN[8][8][3];   // [q][a][j] = dN_a / dxi_j
  float wf[8];
  float Nf[8][8];
  float dNf[8][8][3];
};

// Host-built tables (computed once per process from the closed forms); passed
// to kernels by value as __grid_constant__ parameters.
const RefRule& host_rule(int slot);

// ---------------------------------------------------------------------------
// FP32 -> FP64 without the FP64 pipe.  On GB300 a cvt.f64.f32 issues on the
// FP64 unit (about 0.6 T/s per GPU, the same as DADD), which would make the
// conversion of every accumulated entry cost as much as the assembly itself;
// the widening below is exact and uses integer instructions only.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double f32_to_f64_exact(float x) {
  const uint32_t u = __float_as_uint(x);
  const uint32_t mag = u & 0x7fffffffu;
  if (mag - 0x00800000u < 0x7f000000u) {
    // a normal number: the exponent field moves 3 bits down and its bias
    // grows by 1023 - 127 = 896; the 23 fraction bits split 20 | 3 across
    // the two words
    return __hiloint2double((int)(((mag >> 3) + (896u << 20)) | (u & 0x80000000u)), (int)(u << 29));
  }
  const uint32_t sign = u & 0x80000000u;
  int e = (int)((u >> 23) & 0xffu);
  uint32_t m = u & 0x7fffffu;
  if (e == 0) {
    if (m == 0) return __hiloint2double((int)sign, 0);
    const int lz = __clz((int)m) - 8;  // normalise a subnormal: bring the leading bit to position 23
    m = (m << lz) & 0x7fffffu;
    e = 1 - lz;
  } else if (e == 255) {
    return (double)x;  // inf / nan: keep the IEEE semantics
  }
  const uint32_t hi = sign | ((uint32_t)(e + 896) << 20) | (m >> 3);
  return __hiloint2double((int)hi, (int)(m << 29));
}

// cofactor matrix C of J (J^{-1} = C^T / det J, det J = J_0j C_0j)
__device__ __forceinline__ void cofactors(const double J[3][3], double C[3][3]) {
  C[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  C[0][1] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  C[0][2] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  C[1][0] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
  C[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
  C[1][2] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
  C[2][0] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
  C[2][1] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
  C[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
}

// ---------------------------------------------------------------------------
// Trilinear hex at the 2x2x2 Gauss points in modal form.  With corners in
// binary order p = bx + 2 by + 4 bz (hex8_corner_node maps p to the local node
// order), the map is x(xi) = (1/8) sum_k c_k prod_{s in k} xi_s, where bit s of
// k selects the coordinate xi_s and c_k = sum_p x_p prod_{s in k} sigma_s(p),
// sigma_s(p) = +1 if bit s of p is set, else -1 (a Walsh-Hadamard transform of
// the corner coordinates).  The Jacobian columns are bilinear in the other two
// coordinates, so all eight Jacobians cost 27 FMAs each instead of 63.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int hex8_corner_node(int p) {
  return 4 * (p >> 2) + ((p & 2) ? ((p & 1) ? 2 : 3) : (p & 1));
}

// Lane p of an aligned group of 8 lanes holds the coordinates of corner p on
// entry and c_p on exit (one FP64 add per stage and component: the partner's
// value enters with the sign of the stage).  Every lane of the warp must call it.
// The sign is applied to the partner's value by flipping its sign bit with an
// integer XOR: a per-lane select between v + o and v - o compiles to both FP64
// adds, which doubles the transform's cost on the FP64 pipe.  v + (-o) equals
// v - o exactly (IEEE 754), so the result is unchanged.
__device__ __forceinline__ void hex8_modal(double v[3]) {
  const int p = threadIdx.x & 7;
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    const int bit = 1 << s;
    const int flip = (p & bit) ? (int)0x80000000 : 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const double o = __shfl_xor_sync(0xffffffffu, v[i], bit);
      v[i] += __hiloint2double(__double2hiint(o) ^ flip, __double2loint(o));
    }
  }
}

// J' = 8 J at Gauss point q (xi_s = +-1/sqrt(3) by bit s of q) from the modal
// coefficients c[k][i] of hex8_modal, for the lane's own point, with the work
// shared by the 8 lanes of an element (lane p of an aligned group of 8 holds
// point p; every lane of the warp must call it).  Column j of J' is
// sum_k c_k d(prod_{s in k} xi_s)/d xi_j, four terms; the coordinate products
// are +-1/3 (the rounded square of the point), chosen by sign so that they
// cost no FP64 multiply.  Column 0 depends only on (y, z) and column 1 only
// on (x, z), so each takes 4 distinct values over the 8 points: lanes whose
// bits 0 and 1 agree form column 0, the others column 1, and each lane takes
// the column it lacks from the partner with the same coordinates (lane p ^ 2
// for column 1, p ^ 1 for column 0).  Column 2 depends only on (x, y), shared
// by lanes p and p ^ 4: the lane with bit 2 clear forms its components 0 and
// 1, the other component 2 (twice: the warp issues two slots either way),
// and they exchange: 15 FMAs per lane instead of 27, each entry the same FMA
// chain as a lane forming all of J would evaluate.  SHARE_Z = false forms
// column 2 on every lane (18 FMAs, no selects or shuffles): the block-task
// producers, which are bound by issue rather than by the FP64 unit, measured
// 3.82 against 3.80 ms per 128^3 step with the shared column.
template <bool SHARE_Z = true>
__device__ __forceinline__ void hex8_jacobian_pairs(const double (*c)[3], int q, double J[3][3]) {
  constexpr double g = 0.57735026918962576451;
  constexpr double g2 = g * g;
  const double x = (q & 1) ? g : -g, y = (q & 2) ? g : -g, z = (q & 4) ? g : -g;
  const double xy = ((q ^ (q >> 1)) & 1) ? -g2 : g2;
  const double xz = ((q ^ (q >> 2)) & 1) ? -g2 : g2;
  const double yz = (((q >> 1) ^ (q >> 2)) & 1) ? -g2 : g2;
  const bool first = ((q ^ (q >> 1)) & 1) == 0;  // this lane forms column 0
  const double s = first ? y : x, st = first ? yz : xz;
  const int partner = (int)(threadIdx.x & 31) ^ (first ? 2 : 1);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const double ca = first ? c[1][i] : c[2][i], cc = first ? c[5][i] : c[6][i];
    const double own = fma(c[7][i], st, fma(cc, z, fma(c[3][i], s, ca)));
    const double other = __shfl_sync(0xffffffffu, own, partner);
    J[i][0] = first ? own : other;
    J[i][1] = first ? other : own;
    if constexpr (!SHARE_Z) J[i][2] = fma(c[7][i], xy, fma(c[6][i], y, fma(c[5][i], x, c[4][i])));
  }
  if constexpr (!SHARE_Z) return;
  const bool low = (q & 4) == 0;
  const int zpartner = (int)(threadIdx.x & 31) ^ 4;
  double m[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    // slot u: component u on the low lane, component 2 on the high one
    const double a4 = low ? c[4][u] : c[4][2], a5 = low ? c[5][u] : c[5][2];
    const double a6 = low ? c[6][u] : c[6][2], a7 = low ? c[7][u] : c[7][2];
    m[u] = fma(a7, xy, fma(a6, y, fma(a5, x, a4)));
  }
  const double o0 = __shfl_sync(0xffffffffu, m[0], zpartner), o1 = __shfl_sync(0xffffffffu, m[1], zpartner);
  J[0][2] = low ? m[0] : o0;
  J[1][2] = low ? m[1] : o1;
  J[2][2] = low ? o0 : m[0];
}

// x coordinate at Gauss point q of the 2x2x2 rule from the modal
// coefficients c_k of hex8_modal: (1/8) sum_k c_k prod_{s in k} xi_s, with
// xi_s = +-1/sqrt(3) by bit s of q.  Each weight is (1/8) g^|k| with the sign
// of the product (negative when an odd number of the bits of k are clear in
// q), set by flipping the constant's sign bit with an integer XOR, so the sum
// costs 8 FMAs and no FP64 multiply.  Equal to (1/8) times the sum with the
// weights formed as products of +-g: the powers of g round the same way, and
// the factor 1/8 is exact.
__device__ __forceinline__ double hex8_modal_x(const double (*c)[3], int q) {
  constexpr double g = 0.57735026918962576451;
  constexpr double g2 = g * g, g3 = g2 * g;
  constexpr double mag[8] = {0.125, 0.125 * g, 0.125 * g, 0.125 * g2, 0.125 * g, 0.125 * g2, 0.125 * g2, 0.125 * g3};
  double acc = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int flip = (__popc(k & ~q) & 1) ? (int)0x80000000 : 0;
    acc = fma(c[k][0], __hiloint2double(__double2hiint(mag[k]) ^ flip, __double2loint(mag[k])), acc);
  }
  return acc;
}

// FP64 -> FP32, rounded to nearest even, with integer instructions only
// (IEEE 754 binary64 to binary32).  On GB300 the hardware conversion issues
// on the FP64 unit, and a fallback to it for rare inputs was still issued by
// every warp once the compiler predicated it (ncu: one FP64-pipe instruction
// per conversion beyond the FP64 arithmetic), so no case uses it:
// - a normal result (inline): the 52-bit significand keeps its top 23 bits
//   and rounds up when the 29 dropped bits exceed half an ulp, or equal it
//   with an odd kept part; a carry out of the significand moves into the
//   exponent, which also gives the correct overflow to infinity;
// - a zero or an FP64 subnormal (inline): a zero of the same sign;
// - the rest, in a function of its own so that the common path stays a
//   branch and not predicated code: a subnormal or zero binary32 result (the
//   significand with its leading 1, shifted down to units of 2^-149 and
//   rounded the same way; a carry into bit 23 is the smallest normal number's
//   encoding), overflow to infinity, infinities, and NaNs (quiet, with the top
//   bits of the payload).
static __device__ __noinline__ float f64_to_f32_rare(uint32_t hi, uint32_t lo) {
  const uint32_t sign = hi & 0x80000000u;
  const int Ed = (int)((hi >> 20) & 0x7ffu);
  if (Ed == 0x7ff) {
    const uint32_t payload = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const bool nan = ((hi & 0xfffffu) | lo) != 0u;
    return __uint_as_float(sign | 0x7f800000u | (nan ? (0x00400000u | payload) : 0u));
  }
  const int E = Ed - 896;
  if (E >= 255) return __uint_as_float(sign | 0x7f800000u);
  // value = M 2^(Ed - 1075) with M = 2^52 + fraction; in units of 2^-149 it
  // is M 2^-(30 - E), a shift of at least 30; from 54 on the value is below
  // half a unit and rounds to zero
  const int sh = 30 - E;
  if (sh >= 54) return __uint_as_float(sign);
  const unsigned long long M = (((unsigned long long)(hi & 0xfffffu) | 0x100000ull) << 32) | lo;
  const unsigned long long kept = M >> sh;
  const unsigned long long rest = M & ((1ull << sh) - 1ull);
  const unsigned long long half = 1ull << (sh - 1);
  const uint32_t up = (rest > half) || (rest == half && (kept & 1ull));
  return __uint_as_float(sign | ((uint32_t)kept + up));
}

__device__ __forceinline__ float f64_to_f32_rn(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const int Ed = (int)((hi >> 20) & 0x7ffu);
  const int E = Ed - 896;  // binary32 biased exponent
  if (E > 0 && E < 255) {
    const uint32_t kept = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const uint32_t rest = lo & 0x1fffffffu;
    const uint32_t up = (rest > 0x10000000u) || (rest == 0x10000000u && (kept & 1u));
    return __uint_as_float(((hi & 0x80000000u) | ((uint32_t)E << 23) | kept) + up);
  }
  if (Ed == 0) return __uint_as_float(hi & 0x80000000u);
  return f64_to_f32_rare(hi, lo);
}

// an FP64 value in the tile precision: exact for FP64 tiles, rounded to
// nearest even by integer instructions for FP32 tiles (keeps the FP64 pipe,
// which also runs the hardware conversion, free for the arithmetic)
template <typename R>
__device__ __forceinline__ R to_tile(double x);
template <>
__device__ __forceinline__ double to_tile<double>(double x) {
  return x;
}
template <>
__device__ __forceinline__ float to_tile<float>(double x) {
  return f64_to_f32_rn(x);
}

__device__ __forceinline__ void cofactors(const float J[3][3], float C[3][3]) {
  C[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  C[0][1] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  C[0][2] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  C[1][0] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
  C[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
  C[1][2] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
  C[2][0] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
  C[2][1] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
  C[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
}


// FP64 value of a contribution: exact integer widening of FP32 (keeps the
// FP64 pipe free), identity for FP64
__device__ __forceinline__ double widen(float x) { return f32_to_f64_exact(x); }
__device__ __forceinline__ double widen(double x) { return x; }

// FP64 add into global memory that returns nothing: a reduction carried out
// in L2 on a global-space address (red.global.add.f64), so the warp never
// waits for it.  atomicAdd compiles to that only where the compiler can tell
// the pointer is global; in the persistent kernels, whose pointers come from
// a parameter table indexed at run time, it became a generic-address atomic
// whose result every warp waited for (ncu: no reduction sectors in L2,
// long-scoreboard stalls 4.8 per issue against 1.1 in the per-type kernel).
// A generic-address red behaves the same, hence the explicit conversion.
__device__ __forceinline__ void red_add(double* p, double v) {
  const size_t g = __cvta_generic_to_global(p);
  asm volatile("red.global.add.f64 [%0], %1;" ::"l"(g), "d"(v) : "memory");
}


// add into A or b: FP64 atomic (ATOMIC, Alg. "no coloring"), or a plain
// read-modify-write when no other element of the launch touches the entry
// (COLOR: the launch holds one color class, Alg. "coloring")
template <int SC>
__device__ __forceinline__ void scatter_add(double* p, double v) {
  if constexpr (SC == FEA_SCATTER_ATOMIC)
    red_add(p, v);
  else
    *p += v;
}

}  // namespace fea
