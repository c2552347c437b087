// fea_api.cu -- the C-ABI entry points: errors, mesh upload (element lists
// per type, packed connectivity, map offsets), pattern calls, assemble, check.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "fea_internal.cuh"

namespace fea {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
  return FEA_ERR_CUDA;
}

template <typename T>
static int dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(FEA_ERR_OOM, std::string("cudaMalloc of ") + std::to_string(count * sizeof(T)) +
                                 " bytes failed: " + cudaGetErrorString(e));
  }
  return FEA_OK;
}

static void free_mesh(fea_mesh* m) {
  if (!m) return;
  cudaFree(m->coords);
  cudaFree(m->conn_off);
  cudaFree(m->conn);
  cudaFree(m->map_off);
  for (auto& g : m->group) {
    cudaFree(g.ids);
    cudaFree(g.conn);
    cudaFree(g.mapoff);
  }
  cudaFree(m->status);
  cudaFree(m->rp_node);
  cudaFree(m->col_node);
  cudaFree(m->inc_off);
  cudaFree(m->inc);
  drop_rows_plans(m);
  cudaFree(m->geo[0]);
  cudaFree(m->geo[1]);
  fea::free_sched(m);
  free_color_plan(m);
  free_multidep_plan(m);
  if (m->blocks) {
    free_rows_plan(m->blocks);
    delete m->blocks;
  }
  delete m;
}

#define FEA_TRY(x)                  \
  do {                              \
    int _rc = (x);                  \
    if (_rc != FEA_OK) {            \
      free_mesh(m);                 \
      return _rc;                   \
    }                               \
  } while (0)

static int upload_mesh(const fea_mesh_desc* d, cudaStream_t s, fea_mesh** out) {
  if (!d || !out) return fail(FEA_ERR_ARG, "fea_mesh_upload: null argument");
  *out = nullptr;
  if (d->n_nodes <= 0 || d->n_elems <= 0) return fail(FEA_ERR_ARG, "fea_mesh_upload: empty mesh");
  if (d->n_nodes >= (1ll << 31) || d->n_elems >= (1ll << 31))
    return fail(FEA_ERR_INDEX_OVERFLOW, "fea_mesh_upload: n_nodes and n_elems must be < 2^31");
  if (!d->coords || !d->types || !d->conn_offsets || !d->conn)
    return fail(FEA_ERR_ARG, "fea_mesh_upload: null array");
  const int64_t N = d->n_nodes, E = d->n_elems;

  // host copies of the element arrays (device input is brought back once)
  std::vector<uint8_t> types(E);
  std::vector<int64_t> off(E + 1);
  const uint8_t* ht = d->types;
  const int64_t* ho = d->conn_offsets;
  if (d->on_device) {
    FEA_CUDA(cudaMemcpyAsync(types.data(), d->types, E, cudaMemcpyDeviceToHost, s));
    FEA_CUDA(cudaMemcpyAsync(off.data(), d->conn_offsets, (E + 1) * 8, cudaMemcpyDeviceToHost, s));
    FEA_CUDA(cudaStreamSynchronize(s));
    ht = types.data();
    ho = off.data();
  }
  if (ho[0] != 0) return fail(FEA_ERR_ARG, "fea_mesh_upload: conn_offsets[0] != 0");
  int64_t count[kNumTypes] = {0, 0, 0, 0};
  for (int64_t e = 0; e < E; ++e) {
    int t = ht[e];
    if (t >= kNumTypes) return fail(FEA_ERR_ARG, "fea_mesh_upload: unknown element type at element " + std::to_string(e));
    if (ho[e + 1] - ho[e] != kNodesOf[t])
      return fail(FEA_ERR_ARG, "fea_mesh_upload: conn_offsets does not match the node count of element " +
                                   std::to_string(e));
    count[t]++;
  }
  const int64_t L = ho[E];
  std::vector<int32_t> conn(L);
  if (d->on_device) {
    FEA_CUDA(cudaMemcpyAsync(conn.data(), d->conn, L * 4, cudaMemcpyDeviceToHost, s));
    FEA_CUDA(cudaStreamSynchronize(s));
  } else {
    std::memcpy(conn.data(), d->conn, L * 4);
  }
  for (int64_t t = 0; t < L; ++t)
    if (conn[t] < 0 || conn[t] >= N)
      return fail(FEA_ERR_ARG, "fea_mesh_upload: node id out of range at conn[" + std::to_string(t) + "]");

  fea_mesh* m = new fea_mesh();
  FEA_CUDA(cudaGetDevice(&m->device));
  m->n_nodes = N;
  m->n_elems = E;
  m->conn_len = L;
  int ntypes = 0, last = -1;
  for (int t = 0; t < kNumTypes; ++t)
    if (count[t]) ++ntypes, last = t;
  m->uniform = (ntypes == 1);
  m->uniform_type = m->uniform ? last : -1;

  // map offsets: sum of n_e^2 over preceding elements
  std::vector<int64_t> moff(E + 1);
  moff[0] = 0;
  for (int64_t e = 0; e < E; ++e) moff[e + 1] = moff[e] + (ho[e + 1] - ho[e]) * (ho[e + 1] - ho[e]);
  m->map_len = moff[E];

  FEA_TRY(dalloc(&m->coords, 3 * N));
  FEA_TRY(dalloc(&m->conn_off, E + 1));
  FEA_TRY(dalloc(&m->conn, L));
  FEA_TRY(dalloc(&m->map_off, E + 1));
  FEA_TRY(dalloc(&m->status, 1));
  auto cp = [&](void* dst, const void* src, size_t bytes, bool src_dev) -> int {
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, src_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
    return e == cudaSuccess ? FEA_OK : cuda_fail(e, "cudaMemcpyAsync");
  };
  FEA_TRY(cp(m->coords, d->coords, 3 * N * 8, d->on_device));
  FEA_TRY(cp(m->conn_off, ho, (E + 1) * 8, false));
  FEA_TRY(cp(m->conn, conn.data(), L * 4, false));
  FEA_TRY(cp(m->map_off, moff.data(), (E + 1) * 8, false));
  DevStatus zero = {0, 0, ~0ull};
  FEA_TRY(cp(m->status, &zero, sizeof(zero), false));

  // per-type groups in input order (stable), packed connectivity
  for (int t = 0; t < kNumTypes; ++t) {
    TypeGroup& g = m->group[t];
    g.n = count[t];
    if (!g.n) continue;
    const int nn = kNodesOf[t];
    std::vector<int32_t> ids, pc;
    std::vector<int64_t> mo;
    pc.reserve(g.n * nn);
    if (!m->uniform) {
      ids.reserve(g.n);
      mo.reserve(g.n);
    }
    for (int64_t e = 0; e < E; ++e) {
      if (ht[e] != t) continue;
      for (int a = 0; a < nn; ++a) pc.push_back(conn[ho[e] + a]);
      if (!m->uniform) {
        ids.push_back((int32_t)e);
        mo.push_back(moff[e]);
      }
    }
    FEA_TRY(dalloc(&g.conn, g.n * nn));
    FEA_TRY(cp(g.conn, pc.data(), g.n * nn * 4, false));
    if (!m->uniform) {
      FEA_TRY(dalloc(&g.ids, g.n));
      FEA_TRY(dalloc(&g.mapoff, g.n));
      FEA_TRY(cp(g.ids, ids.data(), g.n * 4, false));
      FEA_TRY(cp(g.mapoff, mo.data(), g.n * 8, false));
    }
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    free_mesh(m);
    return cuda_fail(e, "cudaStreamSynchronize");
  }
  {
    const int rc = init_rule_constants();  // synchronous copy, so never inside a stream capture
    if (rc) {
      free_mesh(m);
      return rc;
    }
  }
  *out = m;
  return FEA_OK;
}

}  // namespace fea

using namespace fea;

extern "C" {

const char* fea_last_error(void) { return fea::g_err.c_str(); }

int fea_abi_version(void) { return FEA_ABI_VERSION; }

int fea_mesh_upload(const fea_mesh_desc* desc, void* stream, fea_mesh** out) {
  return upload_mesh(desc, (cudaStream_t)stream, out);
}

int fea_mesh_set_coords(fea_mesh* m, const double* coords, int on_device, void* stream) {
  if (!m || !coords) return fail(FEA_ERR_ARG, "fea_mesh_set_coords: null argument");
  FEA_CUDA(cudaMemcpyAsync(m->coords, coords, 3 * m->n_nodes * sizeof(double),
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, (cudaStream_t)stream));
  return FEA_OK;
}

int fea_mesh_destroy(fea_mesh* mesh) {
  if (!mesh) return fail(FEA_ERR_ARG, "fea_mesh_destroy: null handle");
  cudaDeviceSynchronize();
  free_mesh(mesh);
  return FEA_OK;
}

int fea_mesh_info(const fea_mesh* m, int64_t* n_nodes, int64_t* n_elems, int64_t* map_len) {
  if (!m) return fail(FEA_ERR_ARG, "fea_mesh_info: null handle");
  if (n_nodes) *n_nodes = m->n_nodes;
  if (n_elems) *n_elems = m->n_elems;
  if (map_len) *map_len = m->map_len;
  return FEA_OK;
}

int fea_pattern_size(fea_mesh* m, int ndof, int64_t* nnz, void* stream) {
  if (!m || !nnz) return fail(FEA_ERR_ARG, "fea_pattern_size: null argument");
  if (ndof != 1 && ndof != 3) return fail(FEA_ERR_ARG, "fea_pattern_size: ndof must be 1 or 3");
  if ((int64_t)ndof * m->n_nodes >= (1ll << 31))
    return fail(FEA_ERR_INDEX_OVERFLOW, "fea_pattern_size: ndof * n_nodes must be < 2^31 (int32 columns)");
  cudaStream_t s = (cudaStream_t)stream;
  if (!m->rp_node) {
    int rc = build_node_graph(m, s);
    if (rc != FEA_OK) return rc;
  }
  m->pattern_ndof = ndof;
  m->pattern_built = false;
  *nnz = (int64_t)ndof * ndof * m->nnz_node;
  return FEA_OK;
}

int fea_build_csr_pattern(fea_mesh* m, int ndof, int64_t* row_ptr, int32_t* col_idx, int32_t* node_map,
                          void* stream) {
  if (!m || !row_ptr) return fail(FEA_ERR_ARG, "fea_build_csr_pattern: null argument");
  if (!m->rp_node || m->pattern_ndof != ndof)
    return fail(FEA_ERR_ARG, "fea_build_csr_pattern: call fea_pattern_size with the same ndof first");
  int rc = write_csr_pattern(m, ndof, row_ptr, col_idx, node_map, (cudaStream_t)stream);
  if (rc == FEA_OK && node_map) m->pattern_built = true;
  return rc;
}

int fea_assemble(const fea_operator* op, fea_mesh* m, const int64_t* row_ptr, const int32_t* node_map,
                 double* A, double* b, void* stream) {
  // rows of complete entry blocks are written with 16-byte stores
  if (((uintptr_t)A & 15u) != 0 || ((uintptr_t)b & 7u) != 0)
    return fail(FEA_ERR_ARG, "fea_assemble: A_vals_d must be 16-byte aligned and b_d 8-byte aligned");
  return fea::assemble(op, m, row_ptr, node_map, A, b, (cudaStream_t)stream);
}

int fea_mesh_set_rows_block(fea_mesh* m, int block_nodes) {
  if (!m) return fail(FEA_ERR_ARG, "fea_mesh_set_rows_block: null handle");
  if (block_nodes < 1 || block_nodes > 512) return fail(FEA_ERR_ARG, "fea_mesh_set_rows_block: block size in [1, 512]");
  if (block_nodes != m->rows_block_nodes) {
    cudaDeviceSynchronize();
    drop_rows_plans(m);
  }
  m->rows_block_nodes = block_nodes;
  return FEA_OK;
}

int fea_mesh_set_block_elems(fea_mesh* m, int block_elems) {
  if (!m) return fail(FEA_ERR_ARG, "fea_mesh_set_block_elems: null handle");
  if (block_elems < 1 || block_elems > kRowsStageHalo)
    return fail(FEA_ERR_ARG, "fea_mesh_set_block_elems: elements per block in [1, " + std::to_string(kRowsStageHalo) + "]");
  if (block_elems != m->block_elems && m->blocks) {
    cudaDeviceSynchronize();
    free_rows_plan(m->blocks);
    delete m->blocks;
    m->blocks = nullptr;
  }
  m->block_elems = block_elems;
  return FEA_OK;
}

int fea_rows_plan_info(const fea_mesh* m, int64_t info[8]) {
  if (!m || !info) return fail(FEA_ERR_ARG, "fea_rows_plan_info: null argument");
  for (int k = 0; k < 8; ++k) info[k] = 0;
  const fea::RowsPlan* pp = m->rows[1] ? m->rows[1] : m->rows[0];
  if (!pp) return FEA_OK;
  const fea::RowsPlan& P = *pp;
  info[0] = P.n_blocks;
  info[1] = P.block_nodes;
  info[2] = P.max_local;
  info[3] = P.max_helem;
  info[4] = P.n_tasks;
  info[5] = P.n_contrib;
  info[6] = P.n_helem_total;
  info[7] = (int64_t)P.bytes;
  return FEA_OK;
}

int fea_color_info(const fea_mesh* m, int32_t* colors_h, int* n_colors) {
  if (!m || !n_colors) return fail(FEA_ERR_ARG, "fea_color_info: null argument");
  if (!m->color) return fail(FEA_ERR_ARG, "fea_color_info: no coloring yet (run a FEA_SCATTER_COLOR assembly)");
  *n_colors = m->color->n_colors;
  if (colors_h) std::memcpy(colors_h, m->color->colors_host.data(), m->n_elems * sizeof(int32_t));
  return FEA_OK;
}

int fea_assemble_launches(const fea_operator* op, const fea_mesh* m, int* n_kernels) {
  return fea::assemble_launches(op, m, n_kernels);
}

int fea_check(fea_mesh* m, void* stream) {
  if (!m) return fail(FEA_ERR_ARG, "fea_check: null handle");
  cudaStream_t s = (cudaStream_t)stream;
  FEA_CUDA(cudaStreamSynchronize(s));
  FEA_CUDA(cudaGetLastError());
  DevStatus st;
  FEA_CUDA(cudaMemcpy(&st, m->status, sizeof(st), cudaMemcpyDeviceToHost));
  if (st.code == 0) return FEA_OK;
  DevStatus zero = {0, 0, ~0ull};
  FEA_CUDA(cudaMemcpy(m->status, &zero, sizeof(zero), cudaMemcpyHostToDevice));
  switch (st.code) {
    case FEA_ERR_INVERTED_ELEMENT:
      return fail(st.code, "inverted element: det J <= 0 at a quadrature point of element " + std::to_string(st.info));
    case FEA_ERR_UNSUPPORTED:
      return fail(st.code, "node " + std::to_string(st.info) +
                               " gathers more than 1024 (element, node) incidences (pattern builder limit)");
    default:
      return fail(st.code, "device error " + std::to_string(st.code) + " (id " + std::to_string(st.info) + ")");
  }
}

}  // extern "C"
