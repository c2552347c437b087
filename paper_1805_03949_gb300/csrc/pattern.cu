// pattern.cu -- the integer CSR pattern / element-to-nonzero map builder.
//
// The sparsity pattern of the assembled system is the node graph of the mesh
// (the local square matrices of Sec. 3.1 of the MPI+X assembly paper): nodes i
// and j couple iff some element holds both, the diagonal included.  It is
// built without a global sort:
//   1. node -> (element, local index) incidence lists (count, scan, fill);
//   2. one warp per node gathers the nodes of its incident elements into
//      shared memory and ranks the distinct ones (rank = number of distinct
//      smaller ids), which gives the sorted row and, for every (element, a, b)
//      incidence, the slot k of node b in row a -- the element-to-nonzero map;
//   3. a scan of the row lengths gives row_ptr; the scalar pattern for ndof
//      interleaved dofs per node is expanded from the node pattern.
// Everything is integer work and deterministic: the atomics of step 1 only
// decide the order of the incidence lists, which no output depends on.
#include <cstdio>
#include <mutex>
#include <string>

#include "fea_internal.cuh"

namespace fea {

constexpr int kMaxCand = 1024;  // (element, node) incidences gathered per node
constexpr int kRowWarps = 4;    // warps per CTA of the row kernel

// ---------------------------------------------------------------------------
// exclusive scan int32 -> int64, out[n] = total (three passes)
// ---------------------------------------------------------------------------
constexpr int kScanBlock = 1024;
constexpr int kScanItems = 4;  // items per thread
constexpr int kScanTile = kScanBlock * kScanItems;

__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t* total) {
  __shared__ int64_t warp_sums[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t w = (lane < (int)(blockDim.x >> 5)) ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    warp_sums[lane] = w;  // inclusive
  }
  __syncthreads();
  int64_t base = warp ? warp_sums[warp - 1] : 0;
  if (total) *total = warp_sums[(blockDim.x >> 5) - 1];
  int64_t r = base + x - v;
  __syncthreads();
  return r;
}

__global__ void k_scan_reduce(const int32_t* in, int64_t n, int64_t* tile_sums) {
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  int64_t s = 0;
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + (int64_t)k * kScanBlock + threadIdx.x;
    if (i < n) s += in[i];
  }
  int64_t tot;
  block_excl_scan(s, &tot);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

__global__ void k_scan_tiles(int64_t* tile_sums, int64_t ntiles) {
  // single CTA: exclusive scan of the tile sums in place, chunk by chunk
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t c = 0; c < ntiles; c += kScanBlock) {
    int64_t i = c + threadIdx.x;
    int64_t v = i < ntiles ? tile_sums[i] : 0;
    int64_t tot;
    int64_t ex = block_excl_scan(v, &tot);
    if (i < ntiles) tile_sums[i] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
}

__global__ void k_scan_apply(const int32_t* in, int64_t n, const int64_t* tile_offsets, int64_t* out) {
  // each thread owns kScanItems consecutive items of the tile
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int32_t v[kScanItems];
  int64_t s = 0;
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0;
    s += v[k];
  }
  int64_t tot;
  int64_t ex = block_excl_scan(s, &tot) + tile_offsets[blockIdx.x];
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = ex;
    ex += v[k];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) out[n] = tile_offsets[blockIdx.x] + tot;
}

int exclusive_scan_i32(const int32_t* in, int64_t n, int64_t* out, cudaStream_t s) {
  int64_t ntiles = (n + kScanTile - 1) / kScanTile;
  if (ntiles < 1) ntiles = 1;
  int64_t* tiles = nullptr;
  FEA_CUDA(cudaMallocAsync(&tiles, ntiles * sizeof(int64_t), s));
  k_scan_reduce<<<(unsigned)ntiles, kScanBlock, 0, s>>>(in, n, tiles);
  k_scan_tiles<<<1, kScanBlock, 0, s>>>(tiles, ntiles);
  k_scan_apply<<<(unsigned)ntiles, kScanBlock, 0, s>>>(in, n, tiles, out);
  FEA_CUDA(cudaGetLastError());
  FEA_CUDA(cudaFreeAsync(tiles, s));
  return FEA_OK;
}

// ---------------------------------------------------------------------------
// node -> incidence lists
// ---------------------------------------------------------------------------
__global__ void k_inc_count(const int32_t* conn, int64_t len, int32_t* cnt) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < len) atomicAdd(&cnt[conn[t]], 1);
}

__global__ void k_inc_fill(const int64_t* conn_off, const int32_t* conn, int64_t n_elems, const int64_t* inc_off,
                           int32_t* cursor, int64_t* inc) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_elems) return;
  for (int64_t t = conn_off[e]; t < conn_off[e + 1]; ++t) {
    int32_t node = conn[t];
    int64_t pos = inc_off[node] + atomicAdd(&cursor[node], 1);
    inc[pos] = e * 16 + (t - conn_off[e]);
  }
}

// ---------------------------------------------------------------------------
// row kernel: one warp per node
//   mode 0: deg[i] = number of distinct neighbours
//   mode 1: col_node[rp[i] + r] = r-th smallest neighbour, node_map entries
// ---------------------------------------------------------------------------
struct RowSmem {
  int32_t cand[kMaxCand];    // gathered neighbour ids
  int32_t flag[kMaxCand];    // first-occurrence flags
  int32_t rank[kMaxCand];    // rank of each first occurrence (-1 otherwise)
  int32_t sorted[kMaxCand];  // the sorted row
  int64_t dst[kMaxCand];     // node_map destination of each candidate
};

__global__ void __launch_bounds__(kRowWarps * 32) k_rows(int mode, int64_t n_nodes, const int64_t* inc_off,
                                                          const int64_t* inc, const int64_t* conn_off,
                                                          const int32_t* conn, const int64_t* map_off,
                                                          int32_t* deg, const int64_t* rp, int32_t* col_node,
                                                          int32_t* node_map, DevStatus* st) {
  extern __shared__ unsigned char smem_raw[];
  RowSmem& S = reinterpret_cast<RowSmem*>(smem_raw)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * kRowWarps + (threadIdx.x >> 5);
  if (i >= n_nodes) return;  // warp-uniform
  const int64_t i0 = inc_off[i], i1 = inc_off[i + 1];

  // gather: candidate list = nodes of every incident element, in incidence order
  int C = 0;
  bool overflow = false;
  for (int64_t t0 = i0; t0 < i1; t0 += 32) {
    int64_t t = t0 + lane;
    int ne = 0;
    int64_t e = 0, a = 0;
    if (t < i1) {
      int64_t v = inc[t];
      e = v >> 4;
      a = v & 15;
      ne = (int)(conn_off[e + 1] - conn_off[e]);
    }
    int x = ne;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    const int start = C + x - ne;
    const int tot = __shfl_sync(0xffffffffu, x, 31);
    if (C + tot > kMaxCand) {  // warp-uniform
      overflow = true;
      break;
    }
    if (t < i1) {
      const int32_t* en = conn + conn_off[e];
      const int64_t mo = map_off[e] + a * ne;
      for (int b = 0; b < ne; ++b) {
        S.cand[start + b] = en[b];
        S.dst[start + b] = mo + b;
      }
    }
    C += tot;
  }
  if (overflow) {
    if (lane == 0) {
      latch_error(st, FEA_ERR_UNSUPPORTED, (unsigned long long)i);
      if (mode == 0) deg[i] = 0;
    }
    return;
  }
  __syncwarp();
  for (int u = lane; u < C; u += 32) {
    const int32_t v = S.cand[u];
    int first = 1;
    for (int w = 0; w < u; ++w)
      if (S.cand[w] == v) {
        first = 0;
        break;
      }
    S.flag[u] = first;
  }
  __syncwarp();
  int mydeg = 0;
  for (int u = lane; u < C; u += 32) {
    int rank = -1;
    if (S.flag[u]) {
      const int32_t v = S.cand[u];
      rank = 0;
      for (int w = 0; w < C; ++w) rank += (S.flag[w] & (S.cand[w] < v));
      ++mydeg;
    }
    S.rank[u] = rank;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mydeg += __shfl_xor_sync(0xffffffffu, mydeg, o);
  if (mode == 0) {
    if (lane == 0) deg[i] = mydeg;
    return;
  }
  __syncwarp();
  for (int u = lane; u < C; u += 32) {
    const int r = S.rank[u];
    if (r >= 0) {
      S.sorted[r] = S.cand[u];
      if (col_node) col_node[rp[i] + r] = S.cand[u];
    }
  }
  __syncwarp();
  if (node_map) {
    for (int u = lane; u < C; u += 32) {
      const int32_t v = S.cand[u];
      int lo = 0, hi = mydeg;  // lower_bound in the sorted row
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (S.sorted[mid] < v)
          lo = mid + 1;
        else
          hi = mid;
      }
      node_map[S.dst[u]] = lo;
    }
  }
}

// ---------------------------------------------------------------------------
// scalar expansion for ndof > 1: one warp per node
// ---------------------------------------------------------------------------
__global__ void k_expand(int64_t n_nodes, int d, const int64_t* rp, const int32_t* col_node, int64_t* row_ptr,
                         int32_t* col_idx) {
  const int lane = threadIdx.x & 31;
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= n_nodes) return;
  const int64_t r0 = rp[i];
  const int64_t deg = rp[i + 1] - r0;
  const int64_t base = (int64_t)d * d * r0;
  if (lane < d) row_ptr[(int64_t)d * i + lane] = base + (int64_t)lane * d * deg;
  if (i == n_nodes - 1 && lane == 0) row_ptr[(int64_t)d * n_nodes] = base + (int64_t)d * d * deg;
  if (!col_idx) return;
  const int64_t tot = (int64_t)d * d * deg;
  for (int64_t t = lane; t < tot; t += 32) {
    // t = c * (d*deg) + d*k + cc
    int64_t rem = t % (d * deg);
    int64_t k = rem / d;
    int cc = (int)(rem % d);
    col_idx[base + t] = d * col_node[r0 + k] + cc;
  }
}

__global__ void k_copy_i64(const int64_t* src, int64_t* dst, int64_t n) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) dst[t] = src[t];
}

static int read_status(fea_mesh* m, cudaStream_t s, int* code, unsigned long long* info) {
  DevStatus st;
  FEA_CUDA(cudaMemcpyAsync(&st, m->status, sizeof(st), cudaMemcpyDeviceToHost, s));
  FEA_CUDA(cudaStreamSynchronize(s));
  *code = st.code;
  *info = st.info;
  return FEA_OK;
}

int build_node_graph(fea_mesh* m, cudaStream_t s) {
  const int64_t N = m->n_nodes, E = m->n_elems, L = m->conn_len;
  int32_t* cnt = nullptr;
  int32_t* cursor = nullptr;
  int32_t* deg = nullptr;
  FEA_CUDA(cudaMalloc(&m->inc_off, (N + 1) * sizeof(int64_t)));
  FEA_CUDA(cudaMalloc(&m->inc, L * sizeof(int64_t)));
  FEA_CUDA(cudaMalloc(&m->rp_node, (N + 1) * sizeof(int64_t)));
  FEA_CUDA(cudaMallocAsync(&cnt, N * sizeof(int32_t), s));
  FEA_CUDA(cudaMallocAsync(&cursor, N * sizeof(int32_t), s));
  FEA_CUDA(cudaMallocAsync(&deg, N * sizeof(int32_t), s));
  FEA_CUDA(cudaMemsetAsync(cnt, 0, N * sizeof(int32_t), s));
  FEA_CUDA(cudaMemsetAsync(cursor, 0, N * sizeof(int32_t), s));
  k_inc_count<<<grid_for(L, 256), 256, 0, s>>>(m->conn, L, cnt);
  int rc = exclusive_scan_i32(cnt, N, m->inc_off, s);
  if (rc) return rc;
  k_inc_fill<<<grid_for(E, 256), 256, 0, s>>>(m->conn_off, m->conn, E, m->inc_off, cursor, m->inc);
  const size_t smem = kRowWarps * sizeof(RowSmem);
  FEA_CUDA(cudaFuncSetAttribute(k_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_rows<<<grid_for(N, kRowWarps), kRowWarps * 32, smem, s>>>(0, N, m->inc_off, m->inc, m->conn_off, m->conn,
                                                               m->map_off, deg, nullptr, nullptr, nullptr,
                                                               m->status);
  rc = exclusive_scan_i32(deg, N, m->rp_node, s);
  if (rc) return rc;
  FEA_CUDA(cudaGetLastError());
  FEA_CUDA(cudaMemcpyAsync(&m->nnz_node, m->rp_node + N, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  int code = 0;
  unsigned long long info = 0;
  rc = read_status(m, s, &code, &info);
  cudaFreeAsync(cnt, s);
  cudaFreeAsync(cursor, s);
  cudaFreeAsync(deg, s);
  if (rc) return rc;
  if (code) {
    DevStatus zero = {0, 0, ~0ull};
    cudaMemcpy(m->status, &zero, sizeof(zero), cudaMemcpyHostToDevice);
    cudaFree(m->rp_node);
    m->rp_node = nullptr;
    return fail(code, "pattern: node " + std::to_string(info) + " gathers more than " + std::to_string(kMaxCand) +
                          " (element, node) incidences");
  }
  FEA_CUDA(cudaMalloc(&m->col_node, (m->nnz_node ? m->nnz_node : 1) * sizeof(int32_t)));
  const size_t smem1 = kRowWarps * sizeof(RowSmem);
  k_rows<<<grid_for(N, kRowWarps), kRowWarps * 32, smem1, s>>>(1, N, m->inc_off, m->inc, m->conn_off, m->conn,
                                                                m->map_off, nullptr, m->rp_node, m->col_node,
                                                                nullptr, m->status);
  FEA_CUDA(cudaGetLastError());
  FEA_CUDA(cudaStreamSynchronize(s));
  return FEA_OK;
}

int write_csr_pattern(fea_mesh* m, int ndof, int64_t* row_ptr, int32_t* col_idx, int32_t* node_map,
                      cudaStream_t s) {
  const int64_t N = m->n_nodes;
  if (node_map) {
    const size_t smem = kRowWarps * sizeof(RowSmem);
    k_rows<<<grid_for(N, kRowWarps), kRowWarps * 32, smem, s>>>(1, N, m->inc_off, m->inc, m->conn_off, m->conn,
                                                                 m->map_off, nullptr, m->rp_node, nullptr,
                                                                 node_map, m->status);
  }
  if (ndof == 1) {
    k_copy_i64<<<grid_for(N + 1, 256), 256, 0, s>>>(m->rp_node, row_ptr, N + 1);
    if (col_idx)
      FEA_CUDA(cudaMemcpyAsync(col_idx, m->col_node, m->nnz_node * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  } else {
    k_expand<<<grid_for(N * 32, 256), 256, 0, s>>>(N, ndof, m->rp_node, m->col_node, row_ptr, col_idx);
  }
  FEA_CUDA(cudaGetLastError());
  return FEA_OK;
}

// ---------------------------------------------------------------------------
// Row pointers from row lengths without any device allocation.
//
// The scan above takes its per-tile partial sums from a stream-ordered
// allocation.  Callers that hand all device memory to their own pool up
// front, or that must not let a library allocate on their behalf, use
// fea_row_ptr_from_counts_noalloc instead: the tile sums live in the
// file-scope array below, which every GPU that loads the library holds until
// the process exits.
// ---------------------------------------------------------------------------
constexpr int64_t kNoAllocMaxTiles = 16384;                      // 128 KB of tile sums
constexpr int64_t kNoAllocMaxCounts = kNoAllocMaxTiles * kScanTile;  // 67,108,864 rows
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) int64_t g_noalloc_tiles[kNoAllocMaxTiles];

static std::mutex g_noalloc_mutex;
static int64_t* g_noalloc_ptr[kNoAllocMaxDevices];  // device address of g_noalloc_tiles, per device

// Device address of the scratch array on the current device: taken once per
// device, with that device current, on the first call there.
static int noalloc_scratch(int64_t** out) {
  int dev = 0;
  FEA_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices)
    return fail(FEA_ERR_UNSUPPORTED, "fea_row_ptr_from_counts_noalloc: device index " + std::to_string(dev) +
                                         " beyond the supported " + std::to_string(kNoAllocMaxDevices));
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_tiles);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_tiles)");
    g_noalloc_ptr[dev] = (int64_t*)p;
  }
  *out = g_noalloc_ptr[dev];
  return FEA_OK;
}

}  // namespace fea

extern "C" int fea_row_ptr_from_counts_noalloc(const int32_t* counts, int64_t n, int64_t* row_ptr, void* stream) {
  using namespace fea;
  if (n < 0 || !row_ptr || (n > 0 && !counts))
    return fail(FEA_ERR_ARG, "fea_row_ptr_from_counts_noalloc: null pointer or negative length");
  if (n > kNoAllocMaxCounts)
    return fail(FEA_ERR_UNSUPPORTED, "fea_row_ptr_from_counts_noalloc: " + std::to_string(n) +
                                         " rows exceed the fixed scratch limit of " +
                                         std::to_string(kNoAllocMaxCounts));
  int64_t* tiles = nullptr;
  int rc = noalloc_scratch(&tiles);
  if (rc != FEA_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  int64_t ntiles = (n + kScanTile - 1) / kScanTile;
  if (ntiles < 1) ntiles = 1;
  // every tile sum read below is written first by k_scan_reduce, so the
  // scratch left by an earlier call needs no clearing
  k_scan_reduce<<<(unsigned)ntiles, kScanBlock, 0, s>>>(counts, n, tiles);
  k_scan_tiles<<<1, kScanBlock, 0, s>>>(tiles, ntiles);
  k_scan_apply<<<(unsigned)ntiles, kScanBlock, 0, s>>>(counts, n, tiles, row_ptr);
  FEA_CUDA(cudaGetLastError());
  return FEA_OK;
}
