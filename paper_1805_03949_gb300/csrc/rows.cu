// rows.cu -- owner-computes assembly of full rows with halo elements.
//
// Sec. 3.1 of the MPI+X assembly paper describes the full-row decomposition:
// nodes (rows) are partitioned into disjoint sets, every subdomain gets all
// the elements that touch its rows ("halo elements", whose work is
// duplicated), and every row comes out fully assembled with no exchange.
// This file applies that decomposition at CTA level on the GPU:
//
//   * nodes are ordered along a Morton (Z-order) space-filling curve -- the
//     SFC partitioner of Sec. 3.2.1 -- and cut greedily into blocks of at most
//     B nodes whose halo fits a shared-memory budget;
//   * a CTA owns one block: it integrates the geometry of every halo element
//     once (scaled gradients in shared memory), then computes each entry block
//     of its rows as a task that gathers its element contributions;
//   * an entry (i, j) with both nodes in the block is computed once and
//     written to row i and, transposed, to row j (the element matrices are
//     symmetric); entries towards nodes of other blocks are computed by both
//     owners (the duplicated halo work of Sec. 3.1);
//   * every entry of A and b is written exactly once, with plain stores: no
//     atomics, no zero fill, bitwise reproducible results.
//
// Per element and quadrature point the CTA keeps g^_a = sqrt(w detJ) grad N_a,
// so one element's contribution to entry block (a, b) is
//   M = sum_q g^_a (x) g^_b,  A^e_ab = lam M + mu M^T + mu tr(M) I   (elasticity)
//   A^e_ab = sum_q k(x_q) g^_a . g^_b                                 (diffusion)
// -- nine FMAs per point for elasticity.
//
// In FEA_FP32_INTEGRATE mode each element's contribution is integrated in
// FP32 and the contributions of an entry are summed as an unevaluated FP32
// pair (error-free TwoSum), then rounded once to FP64 with integer
// instructions; FEA_FP64 computes and sums in FP64.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "element.cuh"
#include "fea_internal.cuh"
#include "rows.cuh"

namespace fea {

// ---------------------------------------------------------------------------
// plan construction (host, once per mesh, ndof and precision)
// ---------------------------------------------------------------------------
static inline uint32_t spread_bits10(uint32_t v) {
  v &= 1023u;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

struct HostBlock {
  std::vector<int32_t> lnodes;     // owned first
  std::vector<int32_t> helem;      // original element ids
  std::vector<uint8_t> htype;
  std::vector<uint16_t> hln;       // [helem][8]
  std::vector<RowTask> tasks;
  std::vector<uint16_t> contrib;
  int n_owned = 0;
};

static int type_of_nn(int nn) { return nn == 4 ? FEA_TET4 : nn == 5 ? FEA_PYR5 : nn == 6 ? FEA_PRISM6 : FEA_HEX8; }

int build_rows_plan(fea_mesh* m, int ndof, int block_nodes, int halo_cap, cudaStream_t s, RowsPlan** out) {
  *out = nullptr;
  if (block_nodes < 1 || block_nodes > kRowsMaxOwned)
    return fail(FEA_ERR_ARG, "rows plan: block size must be in [1, " + std::to_string(kRowsMaxOwned) + "]");
  const int64_t N = m->n_nodes, E = m->n_elems, L = m->conn_len;
  // host copies of the mesh and of the node graph built on the device
  std::vector<double> X(3 * N);
  std::vector<int64_t> coff(E + 1), rp(N + 1), incoff(N + 1), inc(L);
  std::vector<int32_t> conn(L), col(m->nnz_node);
  FEA_CUDA(cudaMemcpyAsync(X.data(), m->coords, 3 * N * 8, cudaMemcpyDeviceToHost, s));
  FEA_CUDA(cudaMemcpyAsync(coff.data(), m->conn_off, (E + 1) * 8, cudaMemcpyDeviceToHost, s));
  FEA_CUDA(cudaMemcpyAsync(conn.data(), m->conn, L * 4, cudaMemcpyDeviceToHost, s));
  FEA_CUDA(cudaMemcpyAsync(rp.data(), m->rp_node, (N + 1) * 8, cudaMemcpyDeviceToHost, s));
  FEA_CUDA(cudaMemcpyAsync(col.data(), m->col_node, m->nnz_node * 4, cudaMemcpyDeviceToHost, s));
  FEA_CUDA(cudaMemcpyAsync(incoff.data(), m->inc_off, (N + 1) * 8, cudaMemcpyDeviceToHost, s));
  FEA_CUDA(cudaMemcpyAsync(inc.data(), m->inc, L * 8, cudaMemcpyDeviceToHost, s));
  FEA_CUDA(cudaStreamSynchronize(s));
  for (int64_t i = 0; i < N; ++i)
    if (rp[i + 1] - rp[i] > 65535)
      return fail(FEA_ERR_UNSUPPORTED, "rows plan: node " + std::to_string(i) + " has more than 65535 neighbours");

  // Morton order of the nodes over their bounding box (10 bits per axis)
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t i = 0; i < N; ++i)
    for (int c = 0; c < 3; ++c) {
      lo[c] = std::min(lo[c], X[3 * i + c]);
      hi[c] = std::max(hi[c], X[3 * i + c]);
    }
  std::vector<uint64_t> key(N);
  for (int64_t i = 0; i < N; ++i) {
    uint32_t q[3];
    for (int c = 0; c < 3; ++c) {
      const double span = hi[c] > lo[c] ? hi[c] - lo[c] : 1.0;
      const double t = (X[3 * i + c] - lo[c]) / span * 1023.0 + 0.5;
      q[c] = (uint32_t)std::min(1023.0, std::max(0.0, t));
    }
    const uint64_t code = spread_bits10(q[0]) | (spread_bits10(q[1]) << 1) | (spread_bits10(q[2]) << 2);
    key[i] = (code << 32) | (uint64_t)i;
  }
  std::sort(key.begin(), key.end());

  // greedy cut of the curve: a block closes at block_nodes nodes, or when the
  // next node would take its halo past halo_cap elements
  std::vector<int64_t> bstart;
  {
    std::vector<int64_t> stamp(E, -1);
    int64_t cur = -1;
    int owned = 0, halo = 0;
    for (int64_t t = 0; t < N; ++t) {
      const int32_t i = (int32_t)(key[t] & 0xffffffffu);
      int add = 0;
      for (int64_t u = incoff[i]; u < incoff[i + 1]; ++u) add += stamp[inc[u] >> 4] != cur;
      if (cur < 0 || owned >= block_nodes || (owned > 0 && halo + add > halo_cap)) {
        cur = (int64_t)bstart.size();
        bstart.push_back(t);
        owned = 0;
        halo = 0;
      }
      for (int64_t u = incoff[i]; u < incoff[i + 1]; ++u) {
        const int64_t e = inc[u] >> 4;
        if (stamp[e] != cur) {
          stamp[e] = cur;
          ++halo;
        }
      }
      ++owned;
    }
    bstart.push_back(N);
  }
  const int64_t nb = (int64_t)bstart.size() - 1;
  std::vector<HostBlock> blocks(nb);

  unsigned nthreads = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  std::vector<std::string> errors(nthreads);
  auto worker = [&](unsigned tid) {
    std::vector<int32_t> local(N, -1);
    std::vector<int32_t> hindex(E, -1);
    std::vector<int32_t> others;
    for (int64_t b = tid; b < nb; b += nthreads) {
      HostBlock& hb = blocks[b];
      for (int64_t t = bstart[b]; t < bstart[b + 1]; ++t) {
        const int32_t i = (int32_t)(key[t] & 0xffffffffu);
        local[i] = (int32_t)hb.lnodes.size();
        hb.lnodes.push_back(i);
      }
      hb.n_owned = (int)hb.lnodes.size();
      for (int li = 0; li < hb.n_owned; ++li) {
        const int32_t i = hb.lnodes[li];
        for (int64_t t = incoff[i]; t < incoff[i + 1]; ++t) {
          const int32_t e = (int32_t)(inc[t] >> 4);
          if (hindex[e] < 0) {
            hindex[e] = 0;  // seen, numbered below
            hb.helem.push_back(e);
          }
        }
      }
      std::sort(hb.helem.begin(), hb.helem.end());
      others.clear();
      for (size_t h = 0; h < hb.helem.size(); ++h) {
        const int32_t e = hb.helem[h];
        hindex[e] = (int32_t)h;
        for (int64_t t = coff[e]; t < coff[e + 1]; ++t)
          if (local[conn[t]] == -1) {
            local[conn[t]] = -2;  // seen, numbered below
            others.push_back(conn[t]);
          }
      }
      std::sort(others.begin(), others.end());
      for (int32_t j : others) {
        local[j] = (int32_t)hb.lnodes.size();
        hb.lnodes.push_back(j);
      }
      if (hb.helem.size() > (size_t)kRowsMaxHalo || hb.lnodes.size() > 65535) {
        errors[tid] = "rows plan: a block touches " + std::to_string(hb.helem.size()) + " elements (limit " +
                      std::to_string(kRowsMaxHalo) + ")";
      }
      hb.htype.resize(hb.helem.size());
      hb.hln.assign(hb.helem.size() * 8, 0);
      for (size_t h = 0; h < hb.helem.size(); ++h) {
        const int32_t e = hb.helem[h];
        const int nn = (int)(coff[e + 1] - coff[e]);
        hb.htype[h] = (uint8_t)type_of_nn(nn);
        for (int a = 0; a < nn; ++a) hb.hln[h * 8 + a] = (uint16_t)local[conn[coff[e] + a]];
      }
      // one task per entry block (i, j) of the owned rows; (i, j) and (j, i) once when both are owned
      for (int li = 0; li < hb.n_owned; ++li) {
        const int32_t i = hb.lnodes[li];
        const int64_t r0 = rp[i], deg = rp[i + 1] - r0;
        for (int64_t k = 0; k < deg; ++k) {
          const int32_t j = col[r0 + k];
          const int32_t lj = local[j];
          RowTask T;
          std::memset(&T, 0, sizeof(T));
          T.li = (uint8_t)li;
          T.lj = (uint16_t)lj;
          T.k = (uint16_t)k;
          T.kt = 0xffff;
          if (lj < hb.n_owned) {
            if (j < i) continue;
            if (j == i) {
              T.flags |= kTaskDiag;
            } else {
              const int32_t* rj = col.data() + rp[j];
              const int64_t dj = rp[j + 1] - rp[j];
              T.kt = (uint16_t)(std::lower_bound(rj, rj + dj, i) - rj);
              T.flags |= kTaskTranspose;
            }
          }
          if (hb.contrib.size() > 65535) errors[tid] = "rows plan: more than 65535 contributions in a block";
          T.coff = (uint16_t)hb.contrib.size();
          int nc = 0;
          for (int64_t t = incoff[i]; t < incoff[i + 1]; ++t) {
            const int32_t e = (int32_t)(inc[t] >> 4);
            const int a = (int)(inc[t] & 15);
            const int nn = (int)(coff[e + 1] - coff[e]);
            for (int bb = 0; bb < nn; ++bb)
              if (conn[coff[e] + bb] == j) {
                hb.contrib.push_back((uint16_t)((hindex[e] << 6) | (a << 3) | bb));
                ++nc;
              }
          }
          if (nc > 255)
            errors[tid] = "rows plan: an entry gathers " + std::to_string(nc) + " element contributions (limit 255)";
          T.nc = (uint8_t)nc;
          hb.tasks.push_back(T);
        }
      }
      // warps take tasks of equal length: order by contributor count, then by row
      std::stable_sort(hb.tasks.begin(), hb.tasks.end(),
                       [](const RowTask& x, const RowTask& y) { return x.nc > y.nc; });
      for (int32_t j : hb.lnodes) local[j] = -1;
      for (int32_t e : hb.helem) hindex[e] = -1;
    }
  };
  std::vector<std::thread> pool;
  for (unsigned t = 0; t < nthreads; ++t) pool.emplace_back(worker, t);
  for (auto& th : pool) th.join();
  for (auto& e : errors)
    if (!e.empty()) return fail(FEA_ERR_UNSUPPORTED, e);

  // flatten
  RowsPlan P;
  P.ndof = ndof;
  P.block_nodes = block_nodes;
  P.halo_cap = halo_cap;
  P.all_hex = m->uniform && m->uniform_type == FEA_HEX8;
  P.n_blocks = nb;
  std::vector<RowBlock> hdr(nb);
  int64_t nl = 0, nh = 0, nt = 0, nc = 0;
  for (int64_t b = 0; b < nb; ++b) {
    const HostBlock& hb = blocks[b];
    RowBlock& H = hdr[b];
    std::memset(&H, 0, sizeof(H));
    H.lnode_off = nl;
    H.helem_off = nh;
    H.task_off = nt;
    H.contrib_off = nc;
    H.n_owned = (uint16_t)hb.n_owned;
    H.n_local = (uint16_t)hb.lnodes.size();
    H.n_helem = (uint16_t)hb.helem.size();
    H.n_tasks = (int32_t)hb.tasks.size();
    // task and contribution lists are padded to 16-byte multiples so that a
    // block's lists start 16-byte aligned for the bulk copy into shared memory
    const int64_t tpad = (hb.tasks.size() + 3) / 4 * 4, cpad = (hb.contrib.size() + 7) / 8 * 8;
    H.task_bytes = (uint32_t)(tpad * sizeof(RowTask));
    H.contrib_bytes = (uint32_t)(cpad * 2);
    nl += hb.lnodes.size();
    nh += hb.helem.size();
    nt += tpad;
    nc += cpad;
    P.max_local = std::max<int>(P.max_local, (int)hb.lnodes.size());
    P.max_helem = std::max<int>(P.max_helem, (int)hb.helem.size());
    P.max_owned = std::max<int>(P.max_owned, hb.n_owned);
    P.max_tasks = std::max<int64_t>(P.max_tasks, tpad);
    P.max_contrib = std::max<int64_t>(P.max_contrib, cpad);
  }
  std::vector<int32_t> lnodes(nl), helem(nh);
  std::vector<uint8_t> htype(nh);
  std::vector<uint16_t> hln(nh * 8), contrib(nc);
  std::vector<RowTask> tasks(nt);
  for (int64_t b = 0; b < nb; ++b) {
    const HostBlock& hb = blocks[b];
    const RowBlock& H = hdr[b];
    std::copy(hb.lnodes.begin(), hb.lnodes.end(), lnodes.begin() + H.lnode_off);
    std::copy(hb.helem.begin(), hb.helem.end(), helem.begin() + H.helem_off);
    std::copy(hb.htype.begin(), hb.htype.end(), htype.begin() + H.helem_off);
    std::copy(hb.hln.begin(), hb.hln.end(), hln.begin() + 8 * H.helem_off);
    std::copy(hb.tasks.begin(), hb.tasks.end(), tasks.begin() + H.task_off);
    std::copy(hb.contrib.begin(), hb.contrib.end(), contrib.begin() + H.contrib_off);
  }
  P.n_tasks = nt;
  P.n_contrib = nc;
  P.n_helem_total = nh;
  auto up = [&](auto** dst, const auto& v) -> int {
    using T = typename std::remove_reference<decltype(v)>::type::value_type;
    const size_t bytes = std::max<size_t>(1, v.size()) * sizeof(T);
    cudaError_t e = cudaMalloc((void**)dst, bytes);
    if (e != cudaSuccess) return fail(FEA_ERR_OOM, "rows plan: cudaMalloc failed");
    P.bytes += bytes;
    if (!v.empty()) {
      e = cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
    }
    return FEA_OK;
  };
  int rc = FEA_OK;
  if (!rc) rc = up(&P.blocks, hdr);
  if (!rc) rc = up(&P.lnodes, lnodes);
  if (!rc) rc = up(&P.helem_id, helem);
  if (!rc) rc = up(&P.helem_type, htype);
  if (!rc) rc = up(&P.helem_ln, hln);
  if (!rc) rc = up(&P.tasks, tasks);
  if (!rc) rc = up(&P.contrib, contrib);
  if (rc) {
    free_rows_plan(&P);
    return rc;
  }
  *out = new RowsPlan(P);
  return FEA_OK;
}

// byte offsets of one block's working set in dynamic shared memory
struct RowsLayout {
  uint32_t X, G, K, W, Dr, rs, tasks, contrib, bar, type, flag, total;
};

static inline uint32_t align_up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

static RowsLayout rows_layout(int precision, int ndof, int max_local, int max_helem, int max_owned,
                              int64_t max_tasks, int64_t max_contrib) {
  const uint32_t r = precision == FEA_FP64 ? 8 : 4;
  RowsLayout L;
  uint32_t o = 0;
  L.X = o;        o += 24u * max_local;
  L.G = o;        o += r * kRowsGStride * max_helem;
  L.K = align_up(o, 8);  o = L.K + r * kRowsQStride * max_helem;
  L.W = align_up(o, 8);  o = L.W + r * kRowsQStride * max_helem;
  L.Dr = align_up(o, 8); o = L.Dr + (precision == FEA_FP64 ? 0u : 4u * kRowsDStride * max_helem);
  L.rs = align_up(o, 8); o = L.rs + 8u * ndof * max_owned;
  L.tasks = align_up(o, 16);   o = L.tasks + (uint32_t)(sizeof(RowTask) * max_tasks);
  L.contrib = align_up(o, 16); o = L.contrib + (uint32_t)(2 * max_contrib);
  L.bar = align_up(o, 8);      o = L.bar + 8;
  L.type = o;                  o += max_helem;
  L.flag = o;                  o += max_helem;
  L.total = align_up(o, 16);
  return L;
}

size_t rows_smem_bytes(int precision, int max_local, int max_helem) {
  // per-element estimate used to choose the halo budget: the working set of
  // one halo element plus its typical share of tasks (7) and contributions (17)
  const RowsLayout L = rows_layout(precision, 3, max_local, max_helem, 0, 7 * max_helem, 17 * max_helem);
  return L.total;
}

int ensure_rows_plan(fea_mesh* m, int ndof, int precision, cudaStream_t s, RowsPlan** out) {
  RowsPlan*& slot = m->rows[precision == FEA_FP64 ? 0 : 1];
  if (slot && slot->ndof == ndof) {
    *out = slot;
    return FEA_OK;
  }
  if (slot) {
    free_rows_plan(slot);
    delete slot;
    slot = nullptr;
  }
  // halo budget so that two CTAs share an SM (about 105 KB each)
  const size_t per_elem = rows_smem_bytes(precision, 0, 1);
  const int halo_cap = (int)((105 * 1024 - 24 * 4 * 64) / per_elem);
  int B = m->rows_block_nodes;
  for (;;) {
    RowsPlan* P = nullptr;
    int rc = build_rows_plan(m, ndof, B, halo_cap, s, &P);
    if (rc == FEA_OK && rows_layout(precision, ndof, P->max_local, P->max_helem, P->max_owned, P->max_tasks,
                                    P->max_contrib).total <= kRowsMaxSmem) {
      slot = P;
      *out = P;
      return FEA_OK;
    }
    if (P) {
      free_rows_plan(P);
      delete P;
    }
    if (rc && rc != FEA_ERR_UNSUPPORTED) return rc;
    if (B <= 1) return rc ? rc : fail(FEA_ERR_UNSUPPORTED, "rows: no block size fits in shared memory");
    B = std::max(1, B / 2);
  }
}

void free_rows_plan(RowsPlan* P) {
  if (!P) return;
  cudaFree(P->blocks);
  cudaFree(P->lnodes);
  cudaFree(P->helem_id);
  cudaFree(P->helem_type);
  cudaFree(P->helem_ln);
  cudaFree(P->tasks);
  cudaFree(P->contrib);
  P->blocks = nullptr;
  P->lnodes = nullptr;
  P->helem_id = nullptr;
  P->helem_type = nullptr;
  P->helem_ln = nullptr;
  P->tasks = nullptr;
  P->contrib = nullptr;
}

void drop_rows_plans(fea_mesh* m) {
  for (auto& p : m->rows)
    if (p) {
      free_rows_plan(p);
      delete p;
      p = nullptr;
    }
}

// ---------------------------------------------------------------------------
// device
// ---------------------------------------------------------------------------
struct RuleSet {
  RefRule r[kNumRules];
};

struct RowsArgs {
  const double* coords;
  const RowBlock* blocks;
  const int32_t* lnodes;
  const int32_t* helem_id;
  const uint8_t* helem_type;
  const uint16_t* helem_ln;
  const RowTask* tasks;
  const uint16_t* contrib;
  const int64_t* row_ptr;
  double* A;
  double* b;
  DevStatus* st;
  int64_t n_blocks;
  int tet_slot;             // kRuleTet1 or kRuleTet4
  int max_local, max_helem;
  RowsLayout L;
  double k0, k2, src, lam, mu, f[3];
};

// --- TMA bulk copy global -> shared with an mbarrier (bounded wait) --------
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of the barrier; gives up after a bounded number of
// polls (each try_wait suspends for a bounded time) and reports false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  for (int it = 0; it < (1 << 22); ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ int slot_of(int type, int tet_slot) {
  return type == FEA_TET4 ? tet_slot : type == FEA_PYR5 ? kRulePyr8 : type == FEA_PRISM6 ? kRulePrism6 : kRuleHex8;
}

__device__ __forceinline__ int nq_of(int type, int tet_slot) {
  return type == FEA_TET4 ? (tet_slot == kRuleTet1 ? 1 : 4) : type == FEA_PRISM6 ? 6 : 8;
}

// shared-memory carve-up of one block's working set
template <typename R>
struct RowsSmem {
  double* X;      // [max_local][3]           node coordinates
  R* G;           // [max_helem][193]         g^_a = sqrt(w detJ) grad N_a, [q][a][3]
  R* K;           // [max_helem][9]           k(x_q) (diffusion)
  R* W;           // [max_helem][9]           w detJ (right-hand side)
  float* Dr;      // [max_helem][23]          FP32 mode: x_a - x_0 (a = 1..7) and x_0 of every element
  int64_t* rs;    // [max_owned][ndof]        row_ptr of the owned rows
  RowTask* tasks; // [max_tasks]              the block's tasks (bulk-copied)
  uint16_t* contrib;  // [max_contrib]        the block's contribution codes (bulk-copied)
  uint64_t* bar;  // mbarrier of the bulk copies
  uint8_t* type;  // [max_helem]
  uint8_t* flag;  // [max_helem]              FP32 mode: distorted -> FP64 geometry
};

template <typename R>
__device__ __forceinline__ RowsSmem<R> carve(unsigned char* base, const RowsLayout& L) {
  RowsSmem<R> sm;
  sm.X = reinterpret_cast<double*>(base + L.X);
  sm.G = reinterpret_cast<R*>(base + L.G);
  sm.K = reinterpret_cast<R*>(base + L.K);
  sm.W = reinterpret_cast<R*>(base + L.W);
  sm.Dr = reinterpret_cast<float*>(base + L.Dr);
  sm.rs = reinterpret_cast<int64_t*>(base + L.rs);
  sm.tasks = reinterpret_cast<RowTask*>(base + L.tasks);
  sm.contrib = reinterpret_cast<uint16_t*>(base + L.contrib);
  sm.bar = reinterpret_cast<uint64_t*>(base + L.bar);
  sm.type = base + L.type;
  sm.flag = base + L.flag;
  return sm;
}

// FP64 geometry of point q of halo element h (nodes through local ids)
template <int OP, int NN, typename R>
__device__ __forceinline__ bool geom64(const RowsSmem<R>& sm, const uint16_t* ln, const RefRule& rr, int h, int q,
                                       const RowsArgs& P) {
  const double* X0 = sm.X + 3 * ln[0];
  double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  double xq = X0[0];
#pragma unroll
  for (int a = 1; a < NN; ++a) {
    const double* Xa = sm.X + 3 * ln[a];
    const double d0 = Xa[0] - X0[0], d1 = Xa[1] - X0[1], d2 = Xa[2] - X0[2];
    xq += rr.N[q][a] * d0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      J[0][j] += d0 * rr.dN[q][a][j];
      J[1][j] += d1 * rr.dN[q][a][j];
      J[2][j] += d2 * rr.dN[q][a][j];
    }
  }
  double C[3][3];
  cofactors(J, C);
  const double det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
  if (!(det > 0.0)) return false;
  const double wd = rr.w[q] * det;
  const double sc = sqrt(wd) / det;  // g^ = sqrt(w detJ) J^{-T} grad_xi N
  R* G = sm.G + (size_t)h * kRowsGStride + q * 24;
#pragma unroll
  for (int a = 0; a < NN; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i)
      G[3 * a + i] = (R)((rr.dN[q][a][0] * C[i][0] + rr.dN[q][a][1] * C[i][1] + rr.dN[q][a][2] * C[i][2]) * sc);
  sm.W[h * kRowsQStride + q] = (R)wd;
  if constexpr (OP == FEA_OP_DIFFUSION) sm.K[h * kRowsQStride + q] = (R)(P.k0 + P.k2 * xq * xq);
  return true;
}

// FP32 geometry on coordinates relative to node 0; false when the element is
// distorted (Frobenius condition number of J above FEA_KAPPA_FP64) or its
// determinant cannot be trusted in FP32 -- the FP64 path then redoes it
template <int OP, int NN>
__device__ __forceinline__ bool geom32(const RowsSmem<float>& sm, const uint16_t* ln, const RefRule& rr, int h, int q,
                                       const RowsArgs& P) {
  (void)ln;
  const float* Dh = sm.Dr + h * kRowsDStride;  // x_a - x_0 rounded once per element (phase 1a)
  float J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  float xr = 0.0f;
#pragma unroll
  for (int a = 1; a < NN; ++a) {
    const float d0 = Dh[3 * (a - 1) + 0], d1 = Dh[3 * (a - 1) + 1], d2 = Dh[3 * (a - 1) + 2];
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
  if (!(det > 0.0f) || !(nj * nc <= kappa2_max * det * det)) return false;
  const float wd = rr.wf[q] * det;
  const float sc = sqrtf(wd) / det;
  float* G = sm.G + (size_t)h * kRowsGStride + q * 24;
#pragma unroll
  for (int a = 0; a < NN; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i)
      G[3 * a + i] = (rr.dNf[q][a][0] * C[i][0] + rr.dNf[q][a][1] * C[i][1] + rr.dNf[q][a][2] * C[i][2]) * sc;
  sm.W[h * kRowsQStride + q] = wd;
  if constexpr (OP == FEA_OP_DIFFUSION) {
    const float x = Dh[21] + xr;
    sm.K[h * kRowsQStride + q] = (float)P.k0 + (float)P.k2 * x * x;
  }
  return true;
}

template <int OP, typename R, bool FP64>
__device__ __forceinline__ bool geom_dispatch(const RowsSmem<R>& sm, const RefRule& rr, const RowsArgs& P,
                                              const uint16_t* ln, int type, int h, int q) {
  if constexpr (FP64 || std::is_same<R, double>::value) {
    switch (type) {
      case FEA_TET4: return geom64<OP, 4>(sm, ln, rr, h, q, P);
      case FEA_PYR5: return geom64<OP, 5>(sm, ln, rr, h, q, P);
      case FEA_PRISM6: return geom64<OP, 6>(sm, ln, rr, h, q, P);
      default: return geom64<OP, 8>(sm, ln, rr, h, q, P);
    }
  } else {
    switch (type) {
      case FEA_TET4: return geom32<OP, 4>(sm, ln, rr, h, q, P);
      case FEA_PYR5: return geom32<OP, 5>(sm, ln, rr, h, q, P);
      case FEA_PRISM6: return geom32<OP, 6>(sm, ln, rr, h, q, P);
      default: return geom32<OP, 8>(sm, ln, rr, h, q, P);
    }
  }
}

// accumulator of one entry: FP64 sums, or FP32 pairs (hi, lo)
template <int PREC>
struct Acc;
template <>
struct Acc<FEA_FP64> {
  double v = 0.0;
  __device__ __forceinline__ void add(double x) { v += x; }
  __device__ __forceinline__ double value() const { return v; }
};
template <>
struct Acc<FEA_FP32_INTEGRATE> {
  float hi = 0.0f, lo = 0.0f;
  __device__ __forceinline__ void add(float x) { two_sum_acc(hi, lo, x); }
  __device__ __forceinline__ double value() const { return ff_to_f64(hi, lo); }
};

// HEX: every halo element is a hex8 with 8 points (compile-time loop bounds)
template <int OP, int PREC, bool HEX>
__global__ void __launch_bounds__(256, 2) k_rows_assemble(const __grid_constant__ RuleSet rules,
                                                          const __grid_constant__ RowsArgs P) {
  using R = typename std::conditional<PREC == FEA_FP64, double, float>::type;
  constexpr int D = OP == FEA_OP_DIFFUSION ? 1 : 3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const RowsSmem<R> sm = carve<R>(smem_raw, P.L);
  if (threadIdx.x == 0) mbar_init(sm.bar);
  __syncthreads();
  uint32_t parity = 0;
  for (int64_t blk = blockIdx.x; blk < P.n_blocks; blk += gridDim.x, parity ^= 1u) {
    const RowBlock H = P.blocks[blk];
    const int32_t* lnodes = P.lnodes + H.lnode_off;
    const uint16_t* hln = P.helem_ln + 8 * (int64_t)H.helem_off;
    // the block's task and contribution lists travel by TMA bulk copy while
    // the geometry phases run (both lists are 16-byte padded and aligned)
    if (threadIdx.x == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // order earlier reads of the buffers
      mbar_expect_tx(sm.bar, H.task_bytes + H.contrib_bytes);
      if (H.task_bytes) bulk_copy_g2s(sm.tasks, P.tasks + H.task_off, H.task_bytes, sm.bar);
      if (H.contrib_bytes) bulk_copy_g2s(sm.contrib, P.contrib + H.contrib_off, H.contrib_bytes, sm.bar);
    }
    // phase 0: node coordinates, element types, owned row starts
    for (int t = threadIdx.x; t < H.n_owned * D; t += blockDim.x)
      sm.rs[t] = P.row_ptr[(int64_t)D * lnodes[t / D] + t % D];
    for (int t = threadIdx.x; t < H.n_local; t += blockDim.x) {
      const int64_t node = lnodes[t];
      sm.X[3 * t + 0] = P.coords[3 * node + 0];
      sm.X[3 * t + 1] = P.coords[3 * node + 1];
      sm.X[3 * t + 2] = P.coords[3 * node + 2];
    }
    for (int t = threadIdx.x; t < H.n_helem; t += blockDim.x) {
      sm.type[t] = HEX ? (uint8_t)FEA_HEX8 : P.helem_type[H.helem_off + t];
      sm.flag[t] = 0;
    }
    __syncthreads();
    if constexpr (PREC != FEA_FP64) {
      // phase 1a: node offsets x_a - x_0 of every element, subtracted in FP64 and
      // rounded to FP32 once per (element, node) rather than per quadrature point
      for (int t = threadIdx.x; t < 8 * H.n_helem; t += blockDim.x) {
        const int h = t >> 3, a = t & 7;
        const int nn = HEX ? 8 : nodes_of(sm.type[h]);
        const double* X0 = sm.X + 3 * hln[8 * h];
        float* Dh = sm.Dr + h * kRowsDStride;
        if (a == 0) {
          Dh[21] = (float)X0[0];
        } else if (a < nn) {
          const double* Xa = sm.X + 3 * hln[8 * h + a];
          Dh[3 * (a - 1) + 0] = (float)(Xa[0] - X0[0]);
          Dh[3 * (a - 1) + 1] = (float)(Xa[1] - X0[1]);
          Dh[3 * (a - 1) + 2] = (float)(Xa[2] - X0[2]);
        }
      }
      __syncthreads();
    }
    // phase 1: geometry of every (halo element, quadrature point)
    for (int t = threadIdx.x; t < 8 * H.n_helem; t += blockDim.x) {
      const int h = t >> 3, q = t & 7;
      const int type = sm.type[h];
      if (!HEX && q >= nq_of(type, P.tet_slot)) continue;
      const RefRule& rr = rules.r[HEX ? (int)kRuleHex8 : slot_of(type, P.tet_slot)];
      bool ok;
      if constexpr (HEX)
        ok = PREC == FEA_FP64 ? geom64<OP, 8>(sm, hln + 8 * h, rr, h, q, P)
                              : geom_dispatch<OP, R, false>(sm, rr, P, hln + 8 * h, FEA_HEX8, h, q);
      else
        ok = geom_dispatch<OP, R, false>(sm, rr, P, hln + 8 * h, type, h, q);
      if (!ok) {
        if constexpr (PREC == FEA_FP64)
          latch_error(P.st, FEA_ERR_INVERTED_ELEMENT, (unsigned long long)P.helem_id[H.helem_off + h]);
        else
          sm.flag[h] = 1;
      }
    }
    if constexpr (PREC != FEA_FP64) {
      __syncthreads();
      for (int t = threadIdx.x; t < 8 * H.n_helem; t += blockDim.x) {
        const int h = t >> 3, q = t & 7;
        const int type = sm.type[h];
        if (!sm.flag[h] || q >= nq_of(type, P.tet_slot)) continue;
        const RefRule& rr = rules.r[slot_of(type, P.tet_slot)];
        if (!geom_dispatch<OP, R, true>(sm, rr, P, hln + 8 * h, type, h, q))
          latch_error(P.st, FEA_ERR_INVERTED_ELEMENT, (unsigned long long)P.helem_id[H.helem_off + h]);
      }
    }
    __syncthreads();
    // phase 2: one task per entry block of the owned rows (lists now in shared memory)
    const bool landed = mbar_wait_bounded(sm.bar, parity);
    if (__syncthreads_or(!landed)) {
      // the copy did not land within the bound: report, wait a last bounded
      // while for the copy in flight, and leave without touching A
      if (threadIdx.x == 0) latch_error(P.st, FEA_ERR_TIMEOUT, (unsigned long long)blk);
      mbar_wait_bounded(sm.bar, parity);
      return;
    }
    const R lam = (R)P.lam, mu = (R)P.mu;
    const uint16_t* cbase = sm.contrib;
    for (int t = threadIdx.x; t < H.n_tasks; t += blockDim.x) {
      const RowTask T = sm.tasks[t];
      Acc<PREC> acc[D][D];
      Acc<PREC> bacc[D];
      const bool diag = T.flags & kTaskDiag;
#pragma unroll 1
      for (int c = 0; c < T.nc; ++c) {
        const int code = cbase[T.coff + c];
        const int h = code >> 6, a = (code >> 3) & 7, bn = code & 7;
        const int type = HEX ? (int)FEA_HEX8 : sm.type[h];
        const int nq = HEX ? 8 : nq_of(type, P.tet_slot);
        const R* ga = sm.G + (size_t)h * kRowsGStride + 3 * a;
        const R* gb = sm.G + (size_t)h * kRowsGStride + 3 * bn;
        R K[D][D];
        if constexpr (OP == FEA_OP_DIFFUSION) {
          R s = R(0);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            if (!HEX && q >= nq) break;
            const R* x = ga + 24 * q;
            const R* y = gb + 24 * q;
            s += sm.K[h * kRowsQStride + q] * (x[0] * y[0] + x[1] * y[1] + x[2] * y[2]);
          }
          K[0][0] = s;
        } else {
          R M[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            if (!HEX && q >= nq) break;
            const R* x = ga + 24 * q;
            const R* y = gb + 24 * q;
            const R x0 = x[0], x1 = x[1], x2 = x[2], y0 = y[0], y1 = y[1], y2 = y[2];
            M[0][0] += x0 * y0; M[0][1] += x0 * y1; M[0][2] += x0 * y2;
            M[1][0] += x1 * y0; M[1][1] += x1 * y1; M[1][2] += x1 * y2;
            M[2][0] += x2 * y0; M[2][1] += x2 * y1; M[2][2] += x2 * y2;
          }
          const R tr = mu * (M[0][0] + M[1][1] + M[2][2]);
#pragma unroll
          for (int c1 = 0; c1 < 3; ++c1)
#pragma unroll
            for (int c2 = 0; c2 < 3; ++c2) K[c1][c2] = lam * M[c1][c2] + mu * M[c2][c1] + (c1 == c2 ? tr : R(0));
        }
#pragma unroll
        for (int c1 = 0; c1 < D; ++c1)
#pragma unroll
          for (int c2 = 0; c2 < D; ++c2) acc[c1][c2].add(K[c1][c2]);
        if (diag) {
          const RefRule& rr = rules.r[HEX ? (int)kRuleHex8 : slot_of(type, P.tet_slot)];
          R rb = R(0);
          for (int q = 0; q < nq; ++q) {
            R Nqa;
            if constexpr (PREC == FEA_FP64)
              Nqa = rr.N[q][a];
            else
              Nqa = rr.Nf[q][a];
            rb += sm.W[h * kRowsQStride + q] * Nqa;
          }
          if constexpr (OP == FEA_OP_DIFFUSION)
            bacc[0].add(rb * (R)P.src);
          else
#pragma unroll
            for (int c1 = 0; c1 < 3; ++c1) bacc[c1].add(rb * (R)P.f[c1]);
        }
      }
      // write the entry block to row i and, transposed, to row j
      double v[D][D];
#pragma unroll
      for (int c1 = 0; c1 < D; ++c1)
#pragma unroll
        for (int c2 = 0; c2 < D; ++c2) v[c1][c2] = acc[c1][c2].value();
      const int64_t gi = lnodes[T.li];
#pragma unroll
      for (int c1 = 0; c1 < D; ++c1) {
        const int64_t base = sm.rs[D * T.li + c1] + (int64_t)D * T.k;
#pragma unroll
        for (int c2 = 0; c2 < D; ++c2) P.A[base + c2] = v[c1][c2];
      }
      if (T.flags & kTaskTranspose) {
#pragma unroll
        for (int c2 = 0; c2 < D; ++c2) {
          const int64_t base = sm.rs[D * T.lj + c2] + (int64_t)D * T.kt;
#pragma unroll
          for (int c1 = 0; c1 < D; ++c1) P.A[base + c1] = v[c1][c2];
        }
      }
      if (diag) {
#pragma unroll
        for (int c1 = 0; c1 < D; ++c1) P.b[D * gi + c1] = bacc[c1].value();
      }
    }
    __syncthreads();
  }
}

int assemble_rows(const fea_operator* op, fea_mesh* m, const int64_t* row_ptr, double* A, double* b,
                  cudaStream_t s, int* launched) {
  const int D = op->kind == FEA_OP_DIFFUSION ? 1 : 3;
  RowsPlan* plan = nullptr;
  int prc = ensure_rows_plan(m, D, op->precision, s, &plan);
  if (prc) return prc;
  const RowsPlan& RP = *plan;
  static RuleSet rules;
  static bool rules_ready = false;
  if (!rules_ready) {
    for (int k = 0; k < kNumRules; ++k) rules.r[k] = host_rule(k);
    rules_ready = true;
  }
  RowsArgs P;
  std::memset(&P, 0, sizeof(P));
  P.coords = m->coords;
  P.blocks = RP.blocks;
  P.lnodes = RP.lnodes;
  P.helem_id = RP.helem_id;
  P.helem_type = RP.helem_type;
  P.helem_ln = RP.helem_ln;
  P.tasks = RP.tasks;
  P.contrib = RP.contrib;
  P.row_ptr = row_ptr;
  P.A = A;
  P.b = b;
  P.st = m->status;
  P.n_blocks = RP.n_blocks;
  P.tet_slot = op->tet_rule ? kRuleTet4 : kRuleTet1;
  P.max_local = RP.max_local;
  P.max_helem = RP.max_helem;
  P.k0 = op->k0;
  P.k2 = op->k2;
  P.src = op->source;
  const double E = op->young, nu = op->poisson;
  P.lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  P.mu = E / (2.0 * (1.0 + nu));
  for (int c = 0; c < 3; ++c) P.f[c] = op->body_force[c];
  P.L = rows_layout(op->precision, D, RP.max_local, RP.max_helem, RP.max_owned, RP.max_tasks, RP.max_contrib);
  const size_t smem = P.L.total;
  if (smem > kRowsMaxSmem)
    return fail(FEA_ERR_UNSUPPORTED, "rows: a block needs " + std::to_string(smem) +
                                         " bytes of shared memory; use a smaller block");
  const unsigned grid = (unsigned)RP.n_blocks;
  auto launch = [&](auto kern) -> int {
    FEA_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, 256, smem, s>>>(rules, P);
    FEA_CUDA(cudaGetLastError());
    return FEA_OK;
  };
  int rc;
  const bool hex = RP.all_hex;
  if (op->kind == FEA_OP_DIFFUSION) {
    if (op->precision == FEA_FP64)
      rc = hex ? launch(k_rows_assemble<FEA_OP_DIFFUSION, FEA_FP64, true>)
               : launch(k_rows_assemble<FEA_OP_DIFFUSION, FEA_FP64, false>);
    else
      rc = hex ? launch(k_rows_assemble<FEA_OP_DIFFUSION, FEA_FP32_INTEGRATE, true>)
               : launch(k_rows_assemble<FEA_OP_DIFFUSION, FEA_FP32_INTEGRATE, false>);
  } else {
    if (op->precision == FEA_FP64)
      rc = hex ? launch(k_rows_assemble<FEA_OP_ELASTICITY, FEA_FP64, true>)
               : launch(k_rows_assemble<FEA_OP_ELASTICITY, FEA_FP64, false>);
    else
      rc = hex ? launch(k_rows_assemble<FEA_OP_ELASTICITY, FEA_FP32_INTEGRATE, true>)
               : launch(k_rows_assemble<FEA_OP_ELASTICITY, FEA_FP32_INTEGRATE, false>);
  }
  if (rc == FEA_OK) *launched = 1;
  return rc;
}

}  // namespace fea
