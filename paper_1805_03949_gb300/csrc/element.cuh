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

}  // namespace fea
