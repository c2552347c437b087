// persistent.cu -- host side of the persistent schedules (sched.cuh): the
// work-item list of a mesh, the scheduling arguments of one launch, and the
// C entry points that expose items and grid sizes to a host-side packer.
#include <algorithm>
#include <cstring>

#include "fea_internal.cuh"

namespace fea {

constexpr int kDefaultChunk = 128;

void free_sched(fea_mesh* m) {
  cudaFree(m->items);
  cudaFree(m->sched_counter);
  cudaFree(m->sched_heads);
  m->items = nullptr;
  m->sched_counter = nullptr;
  m->sched_heads = nullptr;
  m->sched_heads_n = 0;
  m->items_h.clear();
  m->items_chunk = 0;
}

// Items of chunk elements: for each type t in enum order, the group of type t
// (elements of that type in upload order) cut into ceil(n_t / chunk) runs.
static void item_list(const fea_mesh* m, int chunk, std::vector<WorkItem>& out) {
  out.clear();
  for (int t = 0; t < kNumTypes; ++t) {
    const int64_t n = m->group[t].n;
    for (int64_t f = 0; f < n; f += chunk) {
      WorkItem w;
      w.entry = t;
      w.first = (int32_t)f;
      w.count = (int32_t)std::min<int64_t>(chunk, n - f);
      w.pad = 0;
      out.push_back(w);
    }
  }
}

static int ensure_items(fea_mesh* m, int chunk, cudaStream_t s) {
  if (m->items && m->items_chunk == chunk) return FEA_OK;
  std::vector<WorkItem> h;
  item_list(m, chunk, h);
  if (h.size() >= (size_t)INT32_MAX) return fail(FEA_ERR_INDEX_OVERFLOW, "persistent schedule: too many work items");
  cudaFree(m->items);
  m->items = nullptr;
  if (!h.empty()) {
    FEA_CUDA(cudaMalloc(&m->items, h.size() * sizeof(WorkItem)));
    FEA_CUDA(cudaMemcpyAsync(m->items, h.data(), h.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, s));
    FEA_CUDA(cudaStreamSynchronize(s));  // h is a local buffer
  }
  if (!m->sched_counter) FEA_CUDA(cudaMalloc(&m->sched_counter, sizeof(int32_t)));
  m->items_h.swap(h);
  m->items_chunk = chunk;
  return FEA_OK;
}

static int chunk_of(const fea_operator* op) { return op->chunk > 0 ? op->chunk : kDefaultChunk; }

// scheduler state of one persistent launch: items of the operator's chunk,
// the stealing counter and the queue heads, reset on the stream
static int prepare_sched(const fea_operator* op, fea_mesh* m, cudaStream_t s, SchedArgs* S) {
  if (op->chunk < 0 || op->chunk > (1 << 24)) return fail(FEA_ERR_ARG, "fea_assemble: chunk must be in [0, 2^24]");
  const bool queues = op->schedule == FEA_SCHED_QUEUES || op->schedule == FEA_SCHED_QUEUES_STEAL;
  if (queues && (!op->queue_d || !op->queue_off_d || op->n_ctas <= 0))
    return fail(FEA_ERR_ARG, "fea_assemble: the queue schedules need queue_d, queue_off_d and n_ctas > 0");
  if (op->n_ctas < 0) return fail(FEA_ERR_ARG, "fea_assemble: n_ctas must be >= 0");
  int rc = ensure_items(m, chunk_of(op), s);
  if (rc) return rc;
  FEA_CUDA(cudaMemsetAsync(m->sched_counter, 0, sizeof(int32_t), s));
  if (op->schedule == FEA_SCHED_QUEUES_STEAL) {
    if (m->sched_heads_n < op->n_ctas) {
      cudaFree(m->sched_heads);
      m->sched_heads = nullptr;
      m->sched_heads_n = 0;
      FEA_CUDA(cudaMalloc(&m->sched_heads, (size_t)op->n_ctas * sizeof(int32_t)));
      m->sched_heads_n = op->n_ctas;
    }
    FEA_CUDA(cudaMemsetAsync(m->sched_heads, 0, (size_t)op->n_ctas * sizeof(int32_t), s));
  }
  std::memset(S, 0, sizeof(*S));
  S->items = m->items;
  S->n_items = (int32_t)m->items_h.size();
  S->mode = op->schedule;
  S->counter = m->sched_counter;
  S->queue = op->queue_d;
  S->queue_off = op->queue_off_d;
  S->item_ns = op->item_ns_d;
  S->item_cta = op->item_cta_d;
  S->heads = m->sched_heads;
  S->n_queues = op->n_ctas;
  return FEA_OK;
}

int assemble_persistent(const fea_operator* op, fea_mesh* m, const int64_t* row_ptr, const int32_t* node_map,
                        double* A, double* b, cudaStream_t s) {
  if (op->scatter != FEA_SCATTER_ATOMIC)
    return fail(FEA_ERR_UNSUPPORTED, "fea_assemble: the persistent schedules use the ATOMIC scatter");
  const int D = op->kind == FEA_OP_DIFFUSION ? 1 : 3;
  cudaEvent_t* ev = (cudaEvent_t*)op->events;
  const int nev = ev ? op->n_events : 0;
  if (nev > 0) FEA_CUDA(cudaEventRecord(ev[0], s));
  FEA_CUDA(cudaMemsetAsync(A, 0, (size_t)D * D * m->nnz_node * sizeof(double), s));
  FEA_CUDA(cudaMemsetAsync(b, 0, (size_t)m->n_nodes * D * sizeof(double), s));
  SchedArgs S;
  int rc = prepare_sched(op, m, s, &S);
  if (rc) return rc;
  if (nev > 1) FEA_CUDA(cudaEventRecord(ev[1], s));
  if (S.n_items > 0) {
    rc = op->kind == FEA_OP_J2
             ? launch_persistent_j2(op, m, row_ptr, node_map, A, b, S, op->n_ctas, false, s, nullptr)
             : launch_persistent_assemble(op, m, row_ptr, node_map, A, b, S, op->n_ctas, false, s, nullptr);
    if (rc) return rc;
  }
  if (nev > 2) FEA_CUDA(cudaEventRecord(ev[2], s));
  return FEA_OK;
}

int element_loop_persistent(const fea_operator* op, fea_mesh* m, double* stress, cudaStream_t s) {
  cudaEvent_t* ev = (cudaEvent_t*)op->events;
  const int nev = ev ? op->n_events : 0;
  if (nev > 0) FEA_CUDA(cudaEventRecord(ev[0], s));
  SchedArgs S;
  int rc = prepare_sched(op, m, s, &S);
  if (rc) return rc;
  if (nev > 1) FEA_CUDA(cudaEventRecord(ev[1], s));
  if (S.n_items > 0) {
    rc = launch_persistent_j2(op, m, nullptr, nullptr, nullptr, nullptr, S, op->n_ctas, false, s, nullptr, stress,
                              true);
    if (rc) return rc;
  }
  if (nev > 2) FEA_CUDA(cudaEventRecord(ev[2], s));
  return FEA_OK;
}

}  // namespace fea

using namespace fea;

extern "C" {

int fea_work_items(const fea_mesh* m, int chunk, int64_t* n_items, int32_t* type_h, int32_t* first_h,
                   int32_t* count_h) {
  if (!m || !n_items) return fail(FEA_ERR_ARG, "fea_work_items: null argument");
  if (chunk < 0 || chunk > (1 << 24)) return fail(FEA_ERR_ARG, "fea_work_items: chunk must be in [0, 2^24]");
  std::vector<WorkItem> h;
  item_list(m, chunk > 0 ? chunk : kDefaultChunk, h);
  *n_items = (int64_t)h.size();
  for (size_t i = 0; i < h.size(); ++i) {
    if (type_h) type_h[i] = h[i].entry;
    if (first_h) first_h[i] = h[i].first;
    if (count_h) count_h[i] = h[i].count;
  }
  return FEA_OK;
}

int fea_persistent_grid(const fea_operator* op, fea_mesh* m, int* n_ctas) {
  if (!op || !m || !n_ctas) return fail(FEA_ERR_ARG, "fea_persistent_grid: null argument");
  SchedArgs S;
  std::memset(&S, 0, sizeof(S));
  return op->kind == FEA_OP_J2
             ? launch_persistent_j2(op, m, nullptr, nullptr, nullptr, nullptr, S, op->n_ctas, true, nullptr, n_ctas)
             : launch_persistent_assemble(op, m, nullptr, nullptr, nullptr, nullptr, S, op->n_ctas, true, nullptr,
                                          n_ctas);
}

int fea_element_loop_grid(const fea_operator* op, fea_mesh* m, int* n_ctas) {
  if (!op || !m || !n_ctas) return fail(FEA_ERR_ARG, "fea_element_loop_grid: null argument");
  SchedArgs S;
  std::memset(&S, 0, sizeof(S));
  return launch_persistent_j2(op, m, nullptr, nullptr, nullptr, nullptr, S, op->n_ctas, true, nullptr, n_ctas, nullptr,
                              true);
}

}  // extern "C"
