// fea_internal.cuh -- definitions shared by the engine's translation units
// (mesh handle, device status word, error helpers, launch helpers).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "fea_gb300.h"
#include "geometry.cuh"
#include "rows.cuh"
#include "sched.cuh"

namespace fea {

constexpr int kNumTypes = 4;
constexpr int kNodesOf[kNumTypes] = {4, 5, 6, 8};

__host__ __device__ constexpr int nodes_of(int t) {
  return t == FEA_TET4 ? 4 : t == FEA_PYR5 ? 5 : t == FEA_PRISM6 ? 6 : 8;
}

// Device status word latched by kernels; read back by fea_check.
struct DevStatus {
  int code;                 // 0 or a negative fea_status
  int pad;
  unsigned long long info;  // smallest offending element / node id
};

__device__ __forceinline__ void latch_error(DevStatus* st, int code, unsigned long long id) {
  atomicCAS(&st->code, 0, code);
  atomicMin(&st->info, id);
}

// Element coloring (color.cu): group-local element indices per (color, type).
struct ColorPlan {
  int n_colors = 0;
  std::vector<int64_t> seg_off;      // [n_colors * 4 + 1] offsets of the (color, type) segments in lists
  int32_t* lists = nullptr;          // device
  std::vector<int32_t> colors_host;  // color of every element (original ids)
};

// Subdomain plan of FEA_SCATTER_MULTIDEP (multidep.cu): subdomain k is work
// item k of the chunk; its neighbour list (ascending, itself included) names
// the locks it takes; its elements sit in list positions first .. first +
// count of its type, grouped by local color (class c at cb[cb_off[k] + c] ..
// cb[cb_off[k] + c + 1]).
struct MultidepPlan {
  int chunk = 0;
  int64_t n_sub = 0;
  int64_t max_nb = 0;
  int max_colors = 0;
  int held = -1;                        // a lock held in every launch (tests of the bounded wait)
  std::vector<WorkItem> items_h;
  std::vector<int64_t> nb_off_h, cb_off_h;
  std::vector<int32_t> nb_h, order_h, cb_h, color_h;
  std::vector<int32_t> lists_h[4];
  WorkItem* items = nullptr;            // device copies
  int64_t* nb_off = nullptr;
  int32_t* nb = nullptr;
  int32_t* order = nullptr;
  int64_t* cb_off = nullptr;
  int32_t* cb = nullptr;
  int32_t* lists[4] = {nullptr, nullptr, nullptr, nullptr};
  int32_t* state = nullptr;             // [n_sub] 0 pending, 1 taken, 2 done (one allocation with:)
  int32_t* locks = nullptr;             // [n_sub] 0 free
  int32_t* ctrl = nullptr;              // [2] scan hint (priority position), subdomains done
};

// Per-type element group: original ids and packed connectivity.
struct TypeGroup {
  int64_t n = 0;            // elements of this type
  int32_t* ids = nullptr;   // [n] original element ids (nullptr: identity, single-type mesh)
  int32_t* conn = nullptr;  // [n * nodes_of(t)] packed connectivity, local order
  int64_t* mapoff = nullptr;// [n] offset of the element's block in node_map (nullptr: id * nn^2)
};

}  // namespace fea

struct fea_mesh {
  int device = 0;
  int64_t n_nodes = 0;
  int64_t n_elems = 0;
  int64_t conn_len = 0;
  int64_t map_len = 0;
  bool uniform = false;               // one element type, conn_offsets[e] = e * nn
  int uniform_type = -1;
  double* coords = nullptr;           // [3 n_nodes]
  int64_t* conn_off = nullptr;        // [n_elems + 1]
  int32_t* conn = nullptr;            // [conn_len]
  int64_t* map_off = nullptr;         // [n_elems + 1] offsets into node_map
  fea::TypeGroup group[fea::kNumTypes];
  fea::DevStatus* status = nullptr;   // device status word
  // node graph (built by fea_pattern_size)
  int pattern_ndof = 0;               // ndof of the last fea_pattern_size (0: none)
  bool pattern_built = false;         // fea_build_csr_pattern ran for pattern_ndof
  int64_t nnz_node = 0;
  int64_t* rp_node = nullptr;         // [n_nodes + 1]
  int32_t* col_node = nullptr;        // [nnz_node]
  int64_t* inc_off = nullptr;         // [n_nodes + 1] node -> incidences
  int64_t* inc = nullptr;             // [conn_len] incidence = e * 16 + local index
  // owner-computes row assembly (FEA_SCATTER_ROWS)
  fea::RowsPlan* rows[2] = {nullptr, nullptr};  // per precision (FEA_FP64, FEA_FP32_INTEGRATE)
  void* geo[2] = {nullptr, nullptr};            // geometry records per precision (geometry.cu)
  fea::ColorPlan* color = nullptr;              // FEA_SCATTER_COLOR classes (color.cu)
  fea::RowsPlan* blocks = nullptr;              // FEA_SCATTER_BLOCK plan (blocks.cu)
  fea::MultidepPlan* mdep = nullptr;            // FEA_SCATTER_MULTIDEP plan (multidep.cu)
  int block_elems = 64;                         // elements per block of FEA_SCATTER_BLOCK
  int pipe_producer_warps = 6;                  // producer warps of the pipelined block-task kernel (4..8 of 16)
  int rows_block_nodes = 64;
  // persistent schedules (persistent.cu): work items of the last chunk size
  int items_chunk = 0;
  std::vector<fea::WorkItem> items_h;
  fea::WorkItem* items = nullptr;               // device copy of items_h
  int32_t* sched_counter = nullptr;             // FEA_SCHED_STEAL counter
  int32_t* sched_heads = nullptr;               // FEA_SCHED_QUEUES_STEAL queue heads
  int sched_heads_n = 0;
};

namespace fea {

// Thread-local error message.
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define FEA_CUDA(call)                                       \
  do {                                                       \
    cudaError_t _e = (call);                                 \
    if (_e != cudaSuccess) return ::fea::cuda_fail(_e, #call); \
  } while (0)

inline unsigned grid_for(int64_t n, int per_block) {
  int64_t g = (n + per_block - 1) / per_block;
  return (unsigned)(g < 1 ? 1 : g);
}

// pattern.cu
int build_node_graph(fea_mesh* m, cudaStream_t s);
int write_csr_pattern(fea_mesh* m, int ndof, int64_t* row_ptr, int32_t* col_idx, int32_t* node_map,
                      cudaStream_t s);
int exclusive_scan_i32(const int32_t* in, int64_t n, int64_t* out, cudaStream_t s);

// assemble.cu
int assemble(const fea_operator* op, fea_mesh* m, const int64_t* row_ptr, const int32_t* node_map,
             double* A, double* b, cudaStream_t s);
int assemble_launches(const fea_operator* op, const fea_mesh* m, int* n);

// persistent schedules: launchers (assemble.cu, j2.cu) and host side (persistent.cu)
int launch_persistent_assemble(const fea_operator* op, fea_mesh* m, const int64_t* row_ptr, const int32_t* node_map,
                               double* A, double* b, const SchedArgs& S, int n_ctas, bool dry, cudaStream_t s,
                               int* grid_out);
int launch_persistent_j2(const fea_operator* op, fea_mesh* m, const int64_t* row_ptr, const int32_t* node_map,
                         double* A, double* b, const SchedArgs& S, int n_ctas, bool dry, cudaStream_t s,
                         int* grid_out, double* stress = nullptr, bool points_only = false);
int element_loop_persistent(const fea_operator* op, fea_mesh* m, double* stress, cudaStream_t s);
int element_loop_j2(const fea_operator* op, fea_mesh* m, double* stress, cudaStream_t s);
int assemble_persistent(const fea_operator* op, fea_mesh* m, const int64_t* row_ptr, const int32_t* node_map,
                        double* A, double* b, cudaStream_t s);
int assemble_j2(const fea_operator* op, fea_mesh* m, const int64_t* row_ptr, const int32_t* node_map, double* A,
                double* b, cudaStream_t s);
int assemble_nh(const fea_operator* op, fea_mesh* m, const int64_t* row_ptr, const int32_t* node_map, double* A,
                double* b, cudaStream_t s);
int launch_persistent_batch(const fea_operator* op, const void* tab, const int32_t* tab_slot, const SchedArgs& S,
                            int n_ctas, bool dry, cudaStream_t s, int* grid_out);
size_t batch_entry_bytes();
void batch_entry(const fea_operator* op, fea_mesh* m, int t, const int64_t* row_ptr, const int32_t* node_map,
                 double* A, double* b, void* out, int32_t* slot);
int init_rule_constants();     // __constant__ quadrature tables of the persistent kernels (current device)
int init_rule_constants_j2();
void free_sched(fea_mesh* m);

// multidep.cu (host plan) and assemble.cu (its launch)
int ensure_multidep_plan(fea_mesh* m, int chunk, MultidepPlan** out);
void free_multidep_plan(fea_mesh* m);
int reset_multidep(const MultidepPlan& P, cudaStream_t s);
int launch_multidep(const fea_operator* op, fea_mesh* m, const MultidepPlan& plan, const int64_t* row_ptr,
                    const int32_t* node_map, double* A, double* b, cudaStream_t s);

// color.cu
int build_color_plan(fea_mesh* m, cudaStream_t s);
void free_color_plan(fea_mesh* m);
int color_launches(const fea_mesh* m);

}  // namespace fea
