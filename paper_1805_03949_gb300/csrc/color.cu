// color.cu -- element coloring for the FEA_SCATTER_COLOR assembly.
//
// Alg. "coloring" of the MPI+X assembly paper (Sec. 3.2.1): elements are
// colored so that no two elements of one color share a node; each color is
// then assembled without atomics.  The coloring is built once per mesh:
// greedy first-fit on the host, in element order -- an element takes the
// lowest color that no element sharing one of its nodes holds yet (a 64-bit
// mask of the colors at every node) -- which gives the 8 colors of a
// structured hex mesh and few more elsewhere; fewer colors mean fewer and
// larger launches.  A mesh that would need more than 64 colors is colored on
// the GPU by Luby / Jones-Plassmann rounds instead: in round r every
// still-uncolored element whose (hashed, seeded) priority beats all its
// uncolored neighbours takes color r.  Both give a valid coloring by
// construction; the test-suite checks it anyway.  The element lists of each
// (color, type) pair keep the input order, which preserves what spatial
// locality a color class has (the paper notes that coloring loses most of
// it).
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "fea_internal.cuh"

namespace fea {

__device__ __forceinline__ uint32_t color_hash(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return x;
}

__global__ void k_color_round(int round, int64_t n_elems, const int64_t* conn_off, const int32_t* conn,
                              const int64_t* inc_off, const int64_t* inc, int32_t* color, unsigned long long* left) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_elems || color[e] >= 0) return;
  const uint32_t pe = color_hash((uint32_t)e * 2654435761u + 12345u);
  for (int64_t t = conn_off[e]; t < conn_off[e + 1]; ++t) {
    const int32_t node = conn[t];
    for (int64_t u = inc_off[node]; u < inc_off[node + 1]; ++u) {
      const int64_t f = inc[u] >> 4;
      if (f == e) continue;
      const int32_t cf = color[f];
      if (cf >= 0 && cf != round) continue;  // colored in an earlier round
      const uint32_t pf = color_hash((uint32_t)f * 2654435761u + 12345u);
      if (pf > pe || (pf == pe && f > e)) return;  // a neighbour wins this round
    }
  }
  color[e] = round;
  atomicAdd(left, 1ull);
}

// Greedy first-fit in element order (host).  Returns false when an element
// would need a 65th color.
static bool greedy_colors(int64_t E, int64_t N, const std::vector<int64_t>& off, const std::vector<int32_t>& conn,
                          std::vector<int32_t>& color, int* n_colors) {
  std::vector<uint64_t> mask(N, 0);
  int nc = 0;
  for (int64_t e = 0; e < E; ++e) {
    uint64_t used = 0;
    for (int64_t u = off[e]; u < off[e + 1]; ++u) used |= mask[conn[u]];
    if (used == ~0ull) return false;
    const int c = __builtin_ctzll(~used);
    color[e] = c;
    nc = std::max(nc, c + 1);
    for (int64_t u = off[e]; u < off[e + 1]; ++u) mask[conn[u]] |= 1ull << c;
  }
  *n_colors = nc;
  return true;
}

// Luby / Jones-Plassmann rounds on the GPU; *rounds = colors used.
static int jp_colors(fea_mesh* m, cudaStream_t s, std::vector<int32_t>& hc, int* rounds_out) {
  const int64_t E = m->n_elems;
  int32_t* color = nullptr;
  unsigned long long* done = nullptr;
  FEA_CUDA(cudaMalloc(&color, E * sizeof(int32_t)));
  FEA_CUDA(cudaMalloc(&done, sizeof(unsigned long long)));
  FEA_CUDA(cudaMemsetAsync(color, 0xff, E * sizeof(int32_t), s));
  FEA_CUDA(cudaMemsetAsync(done, 0, sizeof(unsigned long long), s));
  unsigned long long colored = 0;
  int rounds = 0;
  const int kMaxRounds = 4096;
  while (colored < (unsigned long long)E && rounds < kMaxRounds) {
    k_color_round<<<grid_for(E, 256), 256, 0, s>>>(rounds, E, m->conn_off, m->conn, m->inc_off, m->inc, color, done);
    FEA_CUDA(cudaGetLastError());
    FEA_CUDA(cudaMemcpyAsync(&colored, done, sizeof(colored), cudaMemcpyDeviceToHost, s));
    FEA_CUDA(cudaStreamSynchronize(s));
    ++rounds;
  }
  if (colored < (unsigned long long)E) {
    cudaFree(color);
    cudaFree(done);
    return fail(FEA_ERR_UNSUPPORTED, "coloring did not finish within " + std::to_string(kMaxRounds) + " rounds");
  }
  hc.resize(E);
  FEA_CUDA(cudaMemcpy(hc.data(), color, E * sizeof(int32_t), cudaMemcpyDeviceToHost));
  cudaFree(color);
  cudaFree(done);
  *rounds_out = rounds;
  return FEA_OK;
}

int build_color_plan(fea_mesh* m, cudaStream_t s) {
  const int64_t E = m->n_elems;
  std::vector<int64_t> off(E + 1);
  std::vector<int32_t> conn(m->conn_len);
  FEA_CUDA(cudaMemcpyAsync(off.data(), m->conn_off, (E + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  FEA_CUDA(cudaMemcpyAsync(conn.data(), m->conn, m->conn_len * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  FEA_CUDA(cudaStreamSynchronize(s));
  std::vector<int32_t> hc(E);
  int rounds = 0;
  if (!greedy_colors(E, m->n_nodes, off, conn, hc, &rounds)) {
    int rc = jp_colors(m, s, hc, &rounds);
    if (rc) return rc;
  }
  // (color, type) segments of group-local indices, input order inside each
  ColorPlan* P = new ColorPlan();
  P->n_colors = rounds;
  std::vector<int64_t> count((size_t)rounds * kNumTypes, 0);
  std::vector<int32_t> gidx(E);
  int64_t next[kNumTypes] = {0, 0, 0, 0};
  std::vector<int> etype(E);
  for (int64_t e = 0; e < E; ++e) {
    const int nn = (int)(off[e + 1] - off[e]);
    const int t = nn == 4 ? FEA_TET4 : nn == 5 ? FEA_PYR5 : nn == 6 ? FEA_PRISM6 : FEA_HEX8;
    etype[e] = t;
    gidx[e] = (int32_t)next[t]++;
    count[(size_t)hc[e] * kNumTypes + t]++;
  }
  P->seg_off.assign(count.size() + 1, 0);
  for (size_t k = 0; k < count.size(); ++k) P->seg_off[k + 1] = P->seg_off[k] + count[k];
  std::vector<int64_t> cursor(P->seg_off.begin(), P->seg_off.end() - 1);
  std::vector<int32_t> lists(E);
  for (int64_t e = 0; e < E; ++e) lists[cursor[(size_t)hc[e] * kNumTypes + etype[e]]++] = gidx[e];
  cudaError_t err = cudaMalloc(&P->lists, std::max<int64_t>(1, E) * sizeof(int32_t));
  if (err != cudaSuccess) {
    delete P;
    return fail(FEA_ERR_OOM, "coloring: cudaMalloc failed");
  }
  FEA_CUDA(cudaMemcpy(P->lists, lists.data(), E * sizeof(int32_t), cudaMemcpyHostToDevice));
  P->colors_host = std::move(hc);
  if (m->color) free_color_plan(m);
  m->color = P;
  return FEA_OK;
}

void free_color_plan(fea_mesh* m) {
  if (!m->color) return;
  cudaFree(m->color->lists);
  delete m->color;
  m->color = nullptr;
}

int color_launches(const fea_mesh* m) {
  if (!m->color) return 0;
  int k = 0;
  for (size_t s = 0; s + 1 < m->color->seg_off.size(); ++s) k += m->color->seg_off[s + 1] > m->color->seg_off[s];
  return k;
}

}  // namespace fea
