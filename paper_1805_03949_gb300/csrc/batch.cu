// batch.cu -- many meshes of uneven sizes through one persistent launch.
//
// A serving-style workload assembles many independent systems at once.  The
// batch holds one parameter-table entry per (mesh, element type) and one work
// item list over all of them; an assembly is two kernels -- a zeroing kernel
// over every A and b (which also resets the scheduler) and one persistent
// launch in which CTAs take items by work stealing, smallest meshes first --
// optionally replayed as one CUDA graph.  Every mesh records the %globaltimer at which its last item
// finished, so per-mesh latencies (completion minus launch start) come out of
// the same run.  The chunk size and the grid are picked by timing candidate
// configurations on the batch itself (fea_batch_autotune).
#include <algorithm>
#include <cstring>
#include <vector>

#include "fea_internal.cuh"

struct fea_batch {
  fea_operator op;
  int n_meshes = 0;
  std::vector<fea_batch_entry> ent;
  void* tab = nullptr;                  // device [4 n][AsmParams]
  int32_t* tab_slot = nullptr;          // device [4 n]
  int chunk = 128;
  int n_ctas = 0;                       // requested (0: resident CTAs)
  int grid = 0;                         // used by the last launch
  std::vector<fea::WorkItem> items_h;
  fea::WorkItem* items = nullptr;
  int32_t* counter = nullptr;
  int32_t* mesh_left = nullptr;         // [n]
  int32_t* mesh_items = nullptr;        // [n] items per mesh (reset value of mesh_left)
  uint64_t* mesh_done = nullptr;        // [n]
  unsigned long long* start = nullptr;  // [1]
  double** zptr = nullptr;              // [2 n] arrays to zero
  int64_t* zlen = nullptr;              // [2 n]
  int64_t zmax = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace fea {

__global__ void __launch_bounds__(256) k_batch_zero(double* const* ptr, const int64_t* len, int n_arr,
                                                    int32_t* mesh_left, const int32_t* mesh_items, int n_meshes,
                                                    int32_t* counter, unsigned long long* start) {
  const int a = blockIdx.y;
  if (a < n_arr) {
    double* p = ptr[a];
    const int64_t n = len[a];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
      p[i] = 0.0;
  }
  if (blockIdx.x == 0 && blockIdx.y == 0) {
    for (int m = threadIdx.x; m < n_meshes; m += blockDim.x) mesh_left[m] = mesh_items[m];
    if (threadIdx.x == 0) {
      *counter = 0;
      *start = ~0ull;
    }
  }
}

static void free_batch(fea_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  cudaFree(b->tab);
  cudaFree(b->tab_slot);
  cudaFree(b->items);
  cudaFree(b->counter);
  cudaFree(b->mesh_left);
  cudaFree(b->mesh_items);
  cudaFree(b->mesh_done);
  cudaFree(b->start);
  cudaFree(b->zptr);
  cudaFree(b->zlen);
  delete b;
}

static void drop_graph(fea_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

// items of every (mesh, type) entry, chunk elements each, mesh by mesh with
// the smallest meshes first: the CTAs take items in list order, so meshes
// complete roughly in that order, and shortest-first minimises the mean
// per-mesh latency without changing the work (ties keep the entry order)
static int build_items(fea_batch* b, int chunk) {
  std::vector<WorkItem> h;
  std::vector<int32_t> per_mesh(b->n_meshes, 0);
  std::vector<int> order(b->n_meshes);
  for (int i = 0; i < b->n_meshes; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return b->ent[x].mesh->n_elems < b->ent[y].mesh->n_elems; });
  for (int i : order)
    for (int t = 0; t < kNumTypes; ++t) {
      const int64_t n = b->ent[i].mesh->group[t].n;
      for (int64_t f = 0; f < n; f += chunk) {
        WorkItem w;
        w.entry = 4 * i + t;
        w.first = (int32_t)f;
        w.count = (int32_t)std::min<int64_t>(chunk, n - f);
        w.pad = 0;
        h.push_back(w);
        ++per_mesh[i];
      }
    }
  if (h.size() >= (size_t)INT32_MAX) return fail(FEA_ERR_INDEX_OVERFLOW, "fea_batch: too many work items");
  cudaFree(b->items);
  b->items = nullptr;
  if (!h.empty()) {
    FEA_CUDA(cudaMalloc(&b->items, h.size() * sizeof(WorkItem)));
    FEA_CUDA(cudaMemcpy(b->items, h.data(), h.size() * sizeof(WorkItem), cudaMemcpyHostToDevice));
  }
  FEA_CUDA(cudaMemcpy(b->mesh_items, per_mesh.data(), per_mesh.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  b->items_h.swap(h);
  b->chunk = chunk;
  drop_graph(b);
  return FEA_OK;
}

static SchedArgs batch_sched(const fea_batch* b) {
  SchedArgs S;
  std::memset(&S, 0, sizeof(S));
  S.items = b->items;
  S.n_items = (int32_t)b->items_h.size();
  S.mode = FEA_SCHED_STEAL;
  S.counter = b->counter;
  S.mesh_left = b->mesh_left;
  S.mesh_done_ns = b->mesh_done;
  S.start_ns = b->start;
  return S;
}

// grid of the persistent launch for the current configuration (no launch)
static int batch_grid(fea_batch* b) {
  const SchedArgs S = batch_sched(b);
  int g = 0;
  const int rc = launch_persistent_batch(&b->op, b->tab, b->tab_slot, S, b->n_ctas, true, nullptr, &g);
  if (rc) return rc;
  b->grid = g;
  return FEA_OK;
}

static int batch_launch(fea_batch* b, cudaStream_t s) {
  const int n_arr = 2 * b->n_meshes;
  const int64_t per = 256 * 16;
  unsigned gx = (unsigned)std::min<int64_t>(std::max<int64_t>((b->zmax + per - 1) / per, 1), 512);
  k_batch_zero<<<dim3(gx, (unsigned)n_arr), 256, 0, s>>>(b->zptr, b->zlen, n_arr, b->mesh_left, b->mesh_items,
                                                         b->n_meshes, b->counter, b->start);
  FEA_CUDA(cudaGetLastError());
  if (b->items_h.empty()) return FEA_OK;
  return launch_persistent_batch(&b->op, b->tab, b->tab_slot, batch_sched(b), b->grid, false, s, nullptr);
}

}  // namespace fea

using namespace fea;

extern "C" {

int fea_batch_create(const fea_operator* op, int n_meshes, const fea_batch_entry* entries_h, fea_batch** out) {
  if (!op || !entries_h || !out || n_meshes < 1 || n_meshes > 32767)
    return fail(FEA_ERR_ARG, "fea_batch_create: bad argument (1 <= n_meshes <= 32767)");
  if (op->kind != FEA_OP_DIFFUSION && op->kind != FEA_OP_ELASTICITY)
    return fail(FEA_ERR_UNSUPPORTED, "fea_batch_create: batches assemble diffusion or elasticity operators");
  if (op->precision != FEA_FP64 && op->precision != FEA_FP32_INTEGRATE && op->precision != FEA_FP32_ADAPTIVE)
    return fail(FEA_ERR_ARG, "fea_batch_create: unknown precision");
  if (op->tet_rule != 0 && op->tet_rule != 1) return fail(FEA_ERR_ARG, "fea_batch_create: tet_rule must be 0 or 1");
  if (op->kind == FEA_OP_ELASTICITY && !(op->poisson > -1.0 && op->poisson < 0.5))
    return fail(FEA_ERR_ARG, "fea_batch_create: poisson must be in (-1, 0.5)");
  if (op->chunk < 0 || op->chunk > (1 << 24) || op->n_ctas < 0)
    return fail(FEA_ERR_ARG, "fea_batch_create: chunk in [0, 2^24] and n_ctas >= 0");
  const int D = op->kind == FEA_OP_DIFFUSION ? 1 : 3;
  for (int i = 0; i < n_meshes; ++i) {
    const fea_batch_entry& e = entries_h[i];
    if (!e.mesh || !e.row_ptr_d || !e.node_map_d || !e.A_d || !e.b_d)
      return fail(FEA_ERR_ARG, "fea_batch_create: null pointer in entry " + std::to_string(i));
    if (e.mesh->pattern_ndof != D || !e.mesh->pattern_built)
      return fail(FEA_ERR_ARG, "fea_batch_create: entry " + std::to_string(i) + " has no pattern for ndof " +
                                   std::to_string(D));
  }
  fea_batch* b = new fea_batch();
  b->op = *op;
  b->op.events = nullptr;
  b->op.n_events = 0;
  b->op.schedule = FEA_SCHED_STEAL;
  b->n_meshes = n_meshes;
  b->ent.assign(entries_h, entries_h + n_meshes);
  b->n_ctas = op->n_ctas;
  const size_t eb = batch_entry_bytes();
  std::vector<unsigned char> tab(eb * 4 * n_meshes);
  std::vector<int32_t> slot(4 * n_meshes);
  std::vector<double*> zp(2 * n_meshes);
  std::vector<int64_t> zl(2 * n_meshes);
  for (int i = 0; i < n_meshes; ++i) {
    const fea_batch_entry& e = entries_h[i];
    for (int t = 0; t < kNumTypes; ++t)
      batch_entry(&b->op, e.mesh, t, e.row_ptr_d, e.node_map_d, e.A_d, e.b_d, tab.data() + eb * (4 * i + t),
                  &slot[4 * i + t]);
    zp[2 * i] = e.A_d;
    zl[2 * i] = (int64_t)D * D * e.mesh->nnz_node;
    zp[2 * i + 1] = e.b_d;
    zl[2 * i + 1] = (int64_t)D * e.mesh->n_nodes;
    b->zmax = std::max(b->zmax, std::max(zl[2 * i], zl[2 * i + 1]));
  }
  auto bail = [&](int rc) {
    free_batch(b);
    return rc;
  };
#define FEA_BATCH_TRY(call)                                  \
  do {                                                       \
    cudaError_t _e = (call);                                 \
    if (_e != cudaSuccess) return bail(cuda_fail(_e, #call)); \
  } while (0)
  FEA_BATCH_TRY(cudaMalloc(&b->tab, tab.size()));
  FEA_BATCH_TRY(cudaMalloc(&b->tab_slot, slot.size() * sizeof(int32_t)));
  FEA_BATCH_TRY(cudaMalloc(&b->counter, sizeof(int32_t)));
  FEA_BATCH_TRY(cudaMalloc(&b->mesh_left, n_meshes * sizeof(int32_t)));
  FEA_BATCH_TRY(cudaMalloc(&b->mesh_items, n_meshes * sizeof(int32_t)));
  FEA_BATCH_TRY(cudaMalloc(&b->mesh_done, n_meshes * sizeof(uint64_t)));
  FEA_BATCH_TRY(cudaMalloc(&b->start, sizeof(unsigned long long)));
  FEA_BATCH_TRY(cudaMalloc(&b->zptr, zp.size() * sizeof(double*)));
  FEA_BATCH_TRY(cudaMalloc(&b->zlen, zl.size() * sizeof(int64_t)));
  FEA_BATCH_TRY(cudaMemcpy(b->tab, tab.data(), tab.size(), cudaMemcpyHostToDevice));
  FEA_BATCH_TRY(cudaMemcpy(b->tab_slot, slot.data(), slot.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  FEA_BATCH_TRY(cudaMemcpy(b->zptr, zp.data(), zp.size() * sizeof(double*), cudaMemcpyHostToDevice));
  FEA_BATCH_TRY(cudaMemcpy(b->zlen, zl.data(), zl.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
  FEA_BATCH_TRY(cudaMemset(b->mesh_done, 0, n_meshes * sizeof(uint64_t)));
#undef FEA_BATCH_TRY
  int rc = build_items(b, op->chunk > 0 ? op->chunk : 128);
  if (!rc) rc = batch_grid(b);
  if (rc) return bail(rc);
  *out = b;
  return FEA_OK;
}

int fea_batch_destroy(fea_batch* b) {
  if (!b) return fail(FEA_ERR_ARG, "fea_batch_destroy: null handle");
  cudaDeviceSynchronize();
  free_batch(b);
  return FEA_OK;
}

int fea_batch_set_config(fea_batch* b, int chunk, int n_ctas) {
  if (!b || chunk < 1 || chunk > (1 << 24) || n_ctas < 0) return fail(FEA_ERR_ARG, "fea_batch_set_config: bad argument");
  FEA_CUDA(cudaDeviceSynchronize());
  if (chunk != b->chunk) {
    int rc = build_items(b, chunk);
    if (rc) return rc;
  }
  if (n_ctas != b->n_ctas) drop_graph(b);
  b->n_ctas = n_ctas;
  return batch_grid(b);
}

int fea_batch_info(const fea_batch* b, int64_t* n_items, int* chunk, int* grid) {
  if (!b) return fail(FEA_ERR_ARG, "fea_batch_info: null handle");
  if (n_items) *n_items = (int64_t)b->items_h.size();
  if (chunk) *chunk = b->chunk;
  if (grid) *grid = b->grid;
  return FEA_OK;
}

int fea_batch_assemble(fea_batch* b, void* stream) {
  if (!b) return fail(FEA_ERR_ARG, "fea_batch_assemble: null handle");
  cudaStream_t s = (cudaStream_t)stream;
  if (b->exec) {
    FEA_CUDA(cudaGraphLaunch(b->exec, s));
    return FEA_OK;
  }
  return batch_launch(b, s);
}

int fea_batch_capture(fea_batch* b, void* stream) {
  if (!b) return fail(FEA_ERR_ARG, "fea_batch_capture: null handle");
  drop_graph(b);
  int rc = batch_grid(b);  // grid and kernel attributes fixed before the capture
  if (rc) return rc;
  cudaStream_t cs = nullptr;
  FEA_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    rc = batch_launch(b, cs);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess && rc == FEA_OK) {
      b->graph = g;
      e = cudaGraphInstantiate(&b->exec, g, 0);
      if (e != cudaSuccess) b->exec = nullptr;
    } else if (g) {
      cudaGraphDestroy(g);
    }
  }
  cudaStreamDestroy(cs);
  if (rc) return rc;
  if (e != cudaSuccess) {
    drop_graph(b);
    return cuda_fail(e, "fea_batch_capture");
  }
  (void)stream;
  return FEA_OK;
}

int fea_batch_latency(fea_batch* b, uint64_t* mesh_ns_h, void* stream) {
  if (!b || !mesh_ns_h) return fail(FEA_ERR_ARG, "fea_batch_latency: null argument");
  FEA_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  std::vector<uint64_t> done(b->n_meshes);
  unsigned long long st = 0;
  FEA_CUDA(cudaMemcpy(done.data(), b->mesh_done, b->n_meshes * sizeof(uint64_t), cudaMemcpyDeviceToHost));
  FEA_CUDA(cudaMemcpy(&st, b->start, sizeof(st), cudaMemcpyDeviceToHost));
  for (int i = 0; i < b->n_meshes; ++i) mesh_ns_h[i] = done[i] > st ? done[i] - st : 0;
  return FEA_OK;
}

int fea_batch_autotune(fea_batch* b, int reps, void* stream, int* chunk_out, int* n_ctas_out, float* ms_out) {
  if (!b || reps < 1) return fail(FEA_ERR_ARG, "fea_batch_autotune: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  FEA_CUDA(cudaGetDevice(&dev));
  FEA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // the resident-CTA grid bounds the candidate grids
  int rc = fea_batch_set_config(b, b->chunk, 0);
  if (rc) return rc;
  const int resident = b->grid;
  const int chunks[] = {16, 32, 64, 128, 256, 512};
  std::vector<int> grids;
  for (int k = 1; k * sms <= resident; ++k) grids.push_back(k * sms);
  if (grids.empty() || grids.back() != resident) grids.push_back(resident);
  cudaEvent_t e0, e1;
  FEA_CUDA(cudaEventCreate(&e0));
  FEA_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_chunk = b->chunk, best_grid = 0;
  for (int c : chunks) {
    for (int g : grids) {
      rc = fea_batch_set_config(b, c, g);
      if (rc) break;
      rc = batch_launch(b, s);  // warm-up
      if (rc) break;
      std::vector<float> t(reps);
      for (int r = 0; r < reps && !rc; ++r) {
        cudaEventRecord(e0, s);
        rc = batch_launch(b, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = fail(FEA_ERR_CUDA, "fea_batch_autotune: event");
        cudaEventElapsedTime(&t[r], e0, e1);
      }
      if (rc) break;
      std::sort(t.begin(), t.end());
      const float med = t[reps / 2];
      if (med < best) {
        best = med;
        best_chunk = c;
        best_grid = g;
      }
    }
    if (rc) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  rc = fea_batch_set_config(b, best_chunk, best_grid);
  if (rc) return rc;
  if (chunk_out) *chunk_out = best_chunk;
  if (n_ctas_out) *n_ctas_out = best_grid;
  if (ms_out) *ms_out = best;
  return FEA_OK;
}

}  // extern "C"
