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
// FP32, widened exactly and summed in FP64; FEA_FP64 computes and sums in FP64.
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
  // element order in every incidence list (filled concurrently on the device):
  // the same contribution order, and so the same FP64 sums, on every build
  for (int64_t i = 0; i < N; ++i) std::sort(inc.begin() + incoff[i], inc.begin() + incoff[i + 1]);
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
      for (size_t h = 0; h < hb.helem.size(); ++h) {
        const int32_t e = hb.helem[h];
        hb.htype[h] = (uint8_t)type_of_nn((int)(coff[e + 1] - coff[e]));
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

  return upload_plan(blocks, ndof, block_nodes, halo_cap, m->uniform && m->uniform_type == FEA_HEX8, out);
}

// Concatenate the per-block lists (16-byte padded) and copy them to the device.
int upload_plan(std::vector<HostBlock>& blocks, int ndof, int block_nodes, int halo_cap, bool all_hex,
                RowsPlan** out) {
  const int64_t nb = (int64_t)blocks.size();
  RowsPlan P;
  P.ndof = ndof;
  P.block_nodes = block_nodes;
  P.halo_cap = halo_cap;
  P.all_hex = all_hex;
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
    const int64_t hpad = (hb.helem.size() + 3) / 4 * 4;
    H.task_bytes = (uint32_t)(tpad * sizeof(RowTask));
    H.contrib_bytes = (uint32_t)(cpad * 2);
    H.helem_bytes = (uint32_t)(hpad * 4);
    nl += hb.lnodes.size();
    nh += hpad;
    nt += tpad;
    nc += cpad;
    P.max_local = std::max<int>(P.max_local, (int)hb.lnodes.size());
    P.max_helem = std::max<int>(P.max_helem, (int)hb.helem.size());
    P.max_helem_padded = std::max<int64_t>(P.max_helem_padded, hpad);
    P.max_owned = std::max<int>(P.max_owned, hb.n_owned);
    P.max_tasks = std::max<int64_t>(P.max_tasks, tpad);
    P.max_contrib = std::max<int64_t>(P.max_contrib, cpad);
  }
  std::vector<int32_t> lnodes(nl), helem(nh);
  std::vector<uint8_t> htype(nh);
  bool with_ln = false;
  for (const HostBlock& hb : blocks) with_ln |= !hb.hln.empty();
  std::vector<uint16_t> hln(with_ln ? nh * 8 : 0);
  std::vector<uint16_t> contrib(nc);
  std::vector<RowTask> tasks(nt);
  for (int64_t b = 0; b < nb; ++b) {
    const HostBlock& hb = blocks[b];
    const RowBlock& H = hdr[b];
    std::copy(hb.lnodes.begin(), hb.lnodes.end(), lnodes.begin() + H.lnode_off);
    std::copy(hb.helem.begin(), hb.helem.end(), helem.begin() + H.helem_off);
    std::copy(hb.htype.begin(), hb.htype.end(), htype.begin() + H.helem_off);
    if (with_ln) std::copy(hb.hln.begin(), hb.hln.end(), hln.begin() + 8 * H.helem_off);
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
  if (!rc && with_ln) rc = up(&P.helem_ln, hln);
  if (!rc) rc = up(&P.tasks, tasks);
  if (!rc) rc = up(&P.contrib, contrib);
  if (rc) {
    free_rows_plan(&P);
    return rc;
  }
  *out = new RowsPlan(P);
  return FEA_OK;
}

static inline uint32_t align_up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

// Shared memory of one block: its owned row starts and node ids (unless
// node_data is false: the pipelined kernel keeps them in its node buffers),
// and the task, contribution and halo-element lists (bulk-copied, 16-byte
// padded); the element records when staged.
RowsLayout rows_layout(const RowsPlan& P, bool stage, int rec_floats, bool node_data) {
  RowsLayout L;
  uint32_t o = 0;
  const uint32_t owned = node_data ? (uint32_t)P.max_owned : 0u;
  L.recs = o;                  o += stage ? (uint32_t)(4 * rec_floats * P.max_helem) : 0u;
  L.rs = align_up(o, 16);      o = L.rs + 8u * P.ndof * owned;
  L.gi = o;                    o += 4u * owned;
  L.tasks = align_up(o, 16);   o = L.tasks + (uint32_t)(sizeof(RowTask) * P.max_tasks);
  L.contrib = align_up(o, 16); o = L.contrib + (uint32_t)(2 * P.max_contrib);
  L.hid = align_up(o, 16);     o = L.hid + (uint32_t)(4 * P.max_helem_padded);
  L.bar = align_up(o, 8);      o = L.bar + 8;
  L.total = align_up(o, 16);
  return L;
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
  // FP32: the halo records are staged in shared memory, so the halo is capped
  // to let two CTAs share an SM; FP64 reads the records through L1 instead
  const bool stage = precision != FEA_FP64;
  const int halo_cap = stage ? kRowsStageHalo : kRowsMaxHalo;
  int B = m->rows_block_nodes;
  for (;;) {
    RowsPlan* P = nullptr;
    int rc = build_rows_plan(m, ndof, B, halo_cap, s, &P);
    if (rc == FEA_OK && rows_layout(*P, stage).total <= kRowsMaxSmem) {
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
  cudaFree(P->zero_runs);
  P->zero_runs = nullptr;
  P->n_zero_runs = 0;
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

}  // namespace fea
