// blocks.cu -- plan of the block-task assembly (FEA_SCATTER_BLOCK).
//
// The local-partitioning and task-based schemes of the MPI+X assembly paper
// (Alg. "local partitioning" and "multideps", Sec. 3.2) cut the element set
// into compact subdomains so that most of the assembly work of a subdomain
// touches only its own entries.  Here a subdomain is a block of at most B
// elements consecutive along a Morton (Z-order) curve of the element
// centroids -- one CTA's work.  Every entry (i, j) that the block's elements
// touch becomes one task whose element contributions are summed in
// registers; the entry is then
//   * stored with a plain store if every element holding both i and j lies
//     in the block (an interior entry: complete), or
//   * added with an FP64 atomic if elements of other blocks add to it as well
//     (a block-boundary entry, resolved globally).
// b and the rows of A that hold boundary entries (those of the nodes whose
// elements lie in more than one block) are zeroed first; every other row of
// A is written whole by stores.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "fea_internal.cuh"
#include "rows.cuh"

namespace fea {

static inline uint32_t spread10(uint32_t v) {
  v &= 1023u;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

int build_blocks_plan(fea_mesh* m, int ndof, int block_elems, cudaStream_t s, RowsPlan** out) {
  *out = nullptr;
  const int64_t N = m->n_nodes, E = m->n_elems, L = m->conn_len;
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
  // the incidence lists are filled concurrently on the device; element order
  // makes each entry's contribution order (its FP64 summation order) the same
  // on every build of the plan
  for (int64_t i = 0; i < N; ++i) std::sort(inc.begin() + incoff[i], inc.begin() + incoff[i + 1]);

  // Morton order of the element centroids
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t i = 0; i < N; ++i)
    for (int c = 0; c < 3; ++c) {
      lo[c] = std::min(lo[c], X[3 * i + c]);
      hi[c] = std::max(hi[c], X[3 * i + c]);
    }
  std::vector<uint64_t> key(E);
  for (int64_t e = 0; e < E; ++e) {
    double cen[3] = {0, 0, 0};
    const int nn = (int)(coff[e + 1] - coff[e]);
    for (int a = 0; a < nn; ++a)
      for (int c = 0; c < 3; ++c) cen[c] += X[3 * (int64_t)conn[coff[e] + a] + c] / nn;
    uint32_t q[3];
    for (int c = 0; c < 3; ++c) {
      const double span = hi[c] > lo[c] ? hi[c] - lo[c] : 1.0;
      q[c] = (uint32_t)std::min(1023.0, std::max(0.0, (cen[c] - lo[c]) / span * 1023.0 + 0.5));
    }
    key[e] = ((uint64_t)(spread10(q[0]) | (spread10(q[1]) << 1) | (spread10(q[2]) << 2)) << 32) | (uint64_t)e;
  }
  std::sort(key.begin(), key.end());

  // greedy cut: at most block_elems elements, at most kRowsMaxOwned distinct nodes
  std::vector<int64_t> bstart;
  {
    std::vector<int64_t> stamp(N, -1);
    int64_t cur = -1;
    int ne = 0, nodes = 0;
    for (int64_t t = 0; t < E; ++t) {
      const int64_t e = (int64_t)(key[t] & 0xffffffffu);
      int add = 0;
      for (int64_t u = coff[e]; u < coff[e + 1]; ++u) add += stamp[conn[u]] != cur;
      if (cur < 0 || ne >= block_elems || nodes + add > kRowsMaxOwned) {
        cur = (int64_t)bstart.size();
        bstart.push_back(t);
        ne = 0;
        nodes = 0;
      }
      for (int64_t u = coff[e]; u < coff[e + 1]; ++u)
        if (stamp[conn[u]] != cur) {
          stamp[conn[u]] = cur;
          ++nodes;
        }
      ++ne;
    }
    bstart.push_back(E);
  }
  const int64_t nb = (int64_t)bstart.size() - 1;
  // the nodes whose elements lie in more than one block, as runs of
  // consecutive ids: only their rows hold entries that several blocks add to
  std::vector<int32_t> zero_runs;
  {
    std::vector<int32_t> blk_of(E);
    for (int64_t b = 0; b < nb; ++b)
      for (int64_t t = bstart[b]; t < bstart[b + 1]; ++t) blk_of[key[t] & 0xffffffffu] = (int32_t)b;
    for (int64_t i = 0; i < N; ++i) {
      bool shared = false;
      for (int64_t u = incoff[i] + 1; u < incoff[i + 1] && !shared; ++u)
        shared = blk_of[inc[u] >> 4] != blk_of[inc[incoff[i]] >> 4];
      if (!shared) continue;
      const size_t r = zero_runs.size();
      if (r && zero_runs[r - 2] + zero_runs[r - 1] == i && zero_runs[r - 1] < kZeroRunNodes)
        ++zero_runs[r - 1];
      else {
        zero_runs.push_back((int32_t)i);
        zero_runs.push_back(1);
      }
    }
  }
  std::vector<HostBlock> blocks(nb);
  unsigned nthreads = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  std::vector<std::string> errors(nthreads);
  auto worker = [&](unsigned tid) {
    std::vector<int32_t> local(N, -1), hindex(E, -1);
    for (int64_t b = tid; b < nb; b += nthreads) {
      HostBlock& hb = blocks[b];
      for (int64_t t = bstart[b]; t < bstart[b + 1]; ++t) hb.helem.push_back((int32_t)(key[t] & 0xffffffffu));
      std::sort(hb.helem.begin(), hb.helem.end());
      for (size_t h = 0; h < hb.helem.size(); ++h) {
        const int32_t e = hb.helem[h];
        hindex[e] = (int32_t)h;
        for (int64_t u = coff[e]; u < coff[e + 1]; ++u)
          if (local[conn[u]] < 0) {
            local[conn[u]] = 0;
            hb.lnodes.push_back(conn[u]);
          }
      }
      std::sort(hb.lnodes.begin(), hb.lnodes.end());
      for (size_t l = 0; l < hb.lnodes.size(); ++l) local[hb.lnodes[l]] = (int32_t)l;
      hb.n_owned = (int)hb.lnodes.size();  // every local node has rows written by this block
      hb.htype.resize(hb.helem.size());
      const bool all_hex = m->uniform && m->uniform_type == FEA_HEX8;
      if (all_hex) hb.hln.assign(hb.helem.size() * 8, 0);
      for (size_t h = 0; h < hb.helem.size(); ++h) {
        const int nn = (int)(coff[hb.helem[h] + 1] - coff[hb.helem[h]]);
        hb.htype[h] = (uint8_t)(nn == 4 ? FEA_TET4 : nn == 5 ? FEA_PYR5 : nn == 6 ? FEA_PRISM6 : FEA_HEX8);
        if (all_hex)  // corner a of block element h is local node hln[8 h + a]
          for (int a = 0; a < 8; ++a) hb.hln[h * 8 + a] = (uint16_t)local[conn[coff[hb.helem[h]] + a]];
      }
      for (int li = 0; li < hb.n_owned; ++li) {
        const int32_t i = hb.lnodes[li];
        bool b_inside = true;  // every element of node i lies in the block
        for (int64_t u = incoff[i]; u < incoff[i + 1]; ++u) b_inside &= hindex[inc[u] >> 4] >= 0;
        const int64_t r0 = rp[i], deg = rp[i + 1] - r0;
        for (int64_t k = 0; k < deg; ++k) {
          const int32_t j = col[r0 + k];
          if (j < i || local[j] < 0) continue;
          RowTask T;
          std::memset(&T, 0, sizeof(T));
          T.li = (uint8_t)li;
          T.lj = (uint16_t)local[j];
          T.k = (uint16_t)k;
          T.kt = 0xffff;
          T.coff = (uint16_t)hb.contrib.size();
          int nc = 0, total = 0;
          for (int64_t u = incoff[i]; u < incoff[i + 1]; ++u) {
            const int64_t e = inc[u] >> 4;
            const int a = (int)(inc[u] & 15);
            for (int64_t v = coff[e]; v < coff[e + 1]; ++v)
              if (conn[v] == j) {
                ++total;
                if (hindex[e] >= 0) {
                  hb.contrib.push_back((uint16_t)((hindex[e] << 6) | (a << 3) | (int)(v - coff[e])));
                  ++nc;
                }
              }
          }
          if (nc == 0) {
            hb.contrib.resize(T.coff);
            continue;  // the block's elements do not touch (i, j)
          }
          if (j == i) {
            T.flags |= kTaskDiag;
            if (!b_inside) T.flags |= kTaskAtomicB;
          } else {
            const int32_t* rj = col.data() + rp[j];
            T.kt = (uint16_t)(std::lower_bound(rj, rj + (rp[j + 1] - rp[j]), i) - rj);
            T.flags |= kTaskTranspose;
          }
          if (nc < total) T.flags |= kTaskAtomicA;
          if (hb.contrib.size() > 65535) errors[tid] = "block plan: more than 65535 contributions in a block";
          T.nc = (uint8_t)std::min(nc, 255);
          if (nc > 255) errors[tid] = "block plan: an entry gathers more than 255 contributions";
          hb.tasks.push_back(T);
        }
      }
      // heaviest tasks first, so that the 32 tasks a warp runs together have
      // about the same number of contributions; within one count the diagonal
      // tasks (which also sum b) come first, so that b's FP64 adds run in
      // warps of diagonal tasks rather than on a few lanes of mixed warps
      std::stable_sort(hb.tasks.begin(), hb.tasks.end(), [](const RowTask& x, const RowTask& y) {
        if (x.nc != y.nc) return x.nc > y.nc;
        return (x.flags & kTaskDiag) > (y.flags & kTaskDiag);
      });
      for (int32_t j : hb.lnodes) local[j] = -1;
      for (int32_t e : hb.helem) hindex[e] = -1;
    }
  };
  std::vector<std::thread> pool;
  for (unsigned t = 0; t < nthreads; ++t) pool.emplace_back(worker, t);
  for (auto& th : pool) th.join();
  for (auto& e : errors)
    if (!e.empty()) return fail(FEA_ERR_UNSUPPORTED, e);
  int rc = upload_plan(blocks, ndof, block_elems, block_elems, m->uniform && m->uniform_type == FEA_HEX8, out);
  if (rc || zero_runs.empty()) return rc;
  RowsPlan* R = *out;
  const size_t zb = zero_runs.size() * sizeof(int32_t);
  if (cudaMalloc((void**)&R->zero_runs, zb) != cudaSuccess ||
      cudaMemcpy(R->zero_runs, zero_runs.data(), zb, cudaMemcpyHostToDevice) != cudaSuccess) {
    free_rows_plan(R);
    delete R;
    *out = nullptr;
    return fail(FEA_ERR_OOM, "block plan: cudaMalloc failed");
  }
  R->n_zero_runs = (int64_t)zero_runs.size() / 2;
  R->bytes += zb;
  return FEA_OK;
}

int ensure_blocks_plan(fea_mesh* m, int ndof, cudaStream_t s, RowsPlan** out) {
  if (m->blocks && m->blocks->ndof == ndof) {
    *out = m->blocks;
    return FEA_OK;
  }
  if (m->blocks) {
    free_rows_plan(m->blocks);
    delete m->blocks;
    m->blocks = nullptr;
  }
  // records of the block's elements are staged in shared memory: the
  // element cap keeps two CTAs per SM
  int B = std::min(m->block_elems, kRowsStageHalo);
  for (;;) {
    RowsPlan* P = nullptr;
    int rc = build_blocks_plan(m, ndof, B, s, &P);
    if (rc == FEA_OK && rows_layout(*P, true).total <= kRowsMaxSmem) {
      m->blocks = P;
      *out = P;
      return FEA_OK;
    }
    if (P) {
      free_rows_plan(P);
      delete P;
    }
    if (rc && rc != FEA_ERR_UNSUPPORTED) return rc;
    if (B <= 1) return rc ? rc : fail(FEA_ERR_UNSUPPORTED, "block plan: no block size fits in shared memory");
    B = std::max(1, B / 2);
  }
}

}  // namespace fea
