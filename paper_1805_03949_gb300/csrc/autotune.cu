// autotune.cu -- the assembly's launch parameters, chosen by timing.
//
// The paper tunes one parameter by hand, the chunk size of its task-based
// assembly (Sec. 5.2: the optimum lies at 100-200 elements per task for its
// meshes).  On the GPU the same role is played by several block and item
// sizes, and the pipelined block-task kernel adds the split of its warps
// between geometry producers and task consumers.  fea_autotune times every
// candidate of the parameters that the operator's scatter and schedule use
// and leaves the mesh (and the operator's chunk) set to the fastest.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "fea_internal.cuh"
#include "rows.cuh"

namespace fea {

namespace {

struct Candidate {
  int block_elems, producer_warps, rows_block_nodes, chunk;
};

// median of reps timed assemblies (after one untimed call, which builds any
// plan the configuration needs)
int time_assembly(fea_operator* op, fea_mesh* m, const int64_t* row_ptr, const int32_t* node_map, double* A,
                  double* b, int reps, cudaStream_t s, float* ms) {
  int rc = fea_assemble(op, m, row_ptr, node_map, A, b, s);
  if (rc) return rc;
  rc = fea_check(m, s);
  if (rc) return rc;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  FEA_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(FEA_ERR_CUDA, "fea_autotune: cudaEventCreate failed");
  }
  std::vector<float> t;
  for (int r = 0; r < reps && rc == FEA_OK; ++r) {
    cudaEventRecord(e0, s);
    rc = fea_assemble(op, m, row_ptr, node_map, A, b, s);
    cudaEventRecord(e1, s);
    if (rc) break;
    cudaError_t e = cudaEventSynchronize(e1);
    float x = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&x, e0, e1);
    if (e != cudaSuccess) rc = cuda_fail(e, "fea_autotune: timing");
    t.push_back(x);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == FEA_OK) rc = fea_check(m, s);
  if (rc) return rc;
  std::sort(t.begin(), t.end());
  *ms = t[t.size() / 2];
  return FEA_OK;
}

int apply(fea_operator* op, fea_mesh* m, const Candidate& c) {
  int rc = fea_mesh_set_block_elems(m, c.block_elems);
  if (!rc) rc = fea_mesh_set_pipe_split(m, c.producer_warps);
  if (!rc) rc = fea_mesh_set_rows_block(m, c.rows_block_nodes);
  op->chunk = c.chunk;
  return rc;
}

}  // namespace

}  // namespace fea

extern "C" {

int fea_mesh_set_pipe_split(fea_mesh* m, int producer_warps) {
  using namespace fea;
  if (!m) return fail(FEA_ERR_ARG, "fea_mesh_set_pipe_split: null handle");
  if (producer_warps < 4 || producer_warps > 8)
    return fail(FEA_ERR_ARG, "fea_mesh_set_pipe_split: producer warps in [4, 8] (of 16)");
  m->pipe_producer_warps = producer_warps;
  return FEA_OK;
}

int fea_autotune(fea_operator* op, fea_mesh* m, const int64_t* row_ptr, const int32_t* node_map, double* A,
                 double* b, int reps, void* stream, fea_tuning* out) {
  using namespace fea;
  if (!op || !m || !row_ptr || !node_map || !A || !b || !out || reps < 1)
    return fail(FEA_ERR_ARG, "fea_autotune: null argument or reps < 1");
  cudaStream_t s = (cudaStream_t)stream;
  const Candidate cur = {m->block_elems, m->pipe_producer_warps, m->rows_block_nodes, op->chunk};
  // the parameters of the path fea_assemble takes for op (in its order)
  std::vector<Candidate> cands;
  const bool plain_op = op->kind == FEA_OP_DIFFUSION || op->kind == FEA_OP_ELASTICITY;
  if (op->scatter == FEA_SCATTER_MULTIDEP) {
    for (int ch : {64, 128, 256}) cands.push_back({cur.block_elems, cur.producer_warps, cur.rows_block_nodes, ch});
  } else if (op->kind != FEA_OP_NEOHOOKE && op->schedule == FEA_SCHED_STEAL) {
    for (int ch : {16, 32, 64, 128, 256})
      cands.push_back({cur.block_elems, cur.producer_warps, cur.rows_block_nodes, ch});
  } else if (plain_op && op->schedule == FEA_SCHED_PER_TYPE && op->scatter == FEA_SCATTER_ROWS) {
    for (int bn : {32, 64, 96, 128}) cands.push_back({cur.block_elems, cur.producer_warps, bn, cur.chunk});
  } else if (plain_op && op->schedule == FEA_SCHED_PER_TYPE && op->scatter == FEA_SCATTER_BLOCK) {
    // the split applies to the pipelined kernel (hex meshes, FP32-integrate)
    const bool pipe = op->precision == FEA_FP32_INTEGRATE && m->uniform && m->uniform_type == FEA_HEX8;
    for (int be : {32, 48, 64, 80})
      for (int pw = 4; pw <= 8; ++pw)
        if (pipe || pw == cur.producer_warps) cands.push_back({be, pw, cur.rows_block_nodes, cur.chunk});
  }
  if (cands.empty()) cands.push_back(cur);
  int best = -1;
  float best_ms = 0.0f;
  for (size_t k = 0; k < cands.size(); ++k) {
    int rc = apply(op, m, cands[k]);
    float ms = 0.0f;
    if (!rc) rc = time_assembly(op, m, row_ptr, node_map, A, b, reps, s, &ms);
    if (rc) {
      apply(op, m, cur);
      return rc;
    }
    if (best < 0 || ms < best_ms) {
      best = (int)k;
      best_ms = ms;
    }
  }
  const Candidate& c = cands[best];
  int rc = apply(op, m, c);
  if (rc) return rc;
  // leave A and b assembled (and any plan built) with the chosen configuration
  rc = fea_assemble(op, m, row_ptr, node_map, A, b, s);
  if (!rc) rc = fea_check(m, s);
  if (rc) return rc;
  out->block_elems = c.block_elems;
  out->producer_warps = c.producer_warps;
  out->rows_block_nodes = c.rows_block_nodes;
  out->chunk = c.chunk;
  out->ms = best_ms;
  out->candidates = (int)cands.size();
  return FEA_OK;
}

}  // extern "C"
