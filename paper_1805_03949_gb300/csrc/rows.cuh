// rows.cuh -- plan of the owner-computes row assembly (see rows.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>
#include <vector>

#include "fea_gb300.h"

namespace fea {

struct DevStatus;

constexpr int kRowsMaxHalo = 1024;            // halo elements per block (10-bit index in a contributor)
constexpr int kRowsMaxOwned = 255;            // owned nodes per block (8-bit index in a task)
constexpr size_t kRowsMaxSmem = 227 * 1024;   // dynamic shared memory of one CTA
constexpr int kRowsGStride = 193;             // values per halo element in the gradient array (8 x 8 x 3 + 1:
                                              // the odd stride spreads consecutive elements over the banks)
constexpr int kRowsQStride = 9;               // values per halo element in the per-point arrays
constexpr int kRowsDStride = 23;              // FP32 relative coordinates per halo element (7 x 3 + x_0 + pad)
constexpr uint8_t kTaskDiag = 1;              // entry (i, i): also accumulates b_i
constexpr uint8_t kTaskTranspose = 2;         // j is owned too: write the transposed block to row j
constexpr uint8_t kTaskAtomicA = 4;           // block-task: elements outside the block add to (i, j) too
constexpr uint8_t kTaskAtomicB = 8;           // block-task: elements outside the block add to b_i too

// One entry block (i, j) of an owned row i: node j sits at slot k of row i
// (and i at slot kt of row j when the transpose is written).  Its element
// contributions are nc codes (halo element << 6 | a << 3 | b) at coff.
struct RowTask {
  uint8_t li, nc, flags, pad;
  uint16_t k, kt, lj, coff;
};
static_assert(sizeof(RowTask) == 12, "RowTask layout");

struct RowBlock {
  int64_t lnode_off, helem_off, task_off, contrib_off;
  uint16_t n_owned, n_local, n_helem, pad;
  int32_t n_tasks;
  uint32_t task_bytes, contrib_bytes, helem_bytes;  // padded list sizes (multiples of 16)
};

// byte offsets of one block's working set in dynamic shared memory
struct RowsLayout {
  uint32_t recs, rs, gi, tasks, contrib, hid, bar, total;
};

constexpr int kRowsRecSmem = 212;     // floats per staged record (208 + 4: 16-byte multiple, spreads banks)
constexpr int kRowsStageHalo = 108;   // halo cap when records are staged (two CTAs per SM)

// Where the values of one staged record sit, in floats from its start:
// gradient g^_a(q)_c at q * Q + 3 a + c, the weight w det J at W + q, k(x_q)
// at K + q; records follow one another every S floats.
template <int Q, int W, int K, int S>
struct RecLayout {
  static constexpr int q = Q, w = W, k = K, stride = S;
};
// the layout of the geometry pass's global records (bulk-copied as they are)
using RecCopied = RecLayout<24, 192, 200, kRowsRecSmem>;
// records computed in shared memory by the pipelined block-task kernel.  The
// strides were chosen with a model of the kernel's shared-memory accesses on
// a 4 x 4 x 4 hex block (its 1,161 tasks in the order the plan gives them, the
// 32 lanes of each consumer warp reading g^_a(q) and g^_b(q) of their
// contributions, and the producer warps' stores): point stride 28 and record
// stride 251 need 7,480 wavefronts per block against 11,192 for the copied
// layout (24, 212); 216 floats per record, the smallest 16-byte multiple,
// would need 16,784
using RecPipe = RecLayout<28, 224, 232, 251>;

struct RowsPlan {
  int ndof = 0;
  int block_nodes = 0;      // cap on owned nodes per block
  int halo_cap = 0;         // cap on halo elements per block (a single node may exceed it)
  bool all_hex = false;     // every element is a hex8: the kernel specialised for it applies
  int64_t n_blocks = 0;
  int max_local = 0, max_helem = 0, max_owned = 0;
  int64_t max_tasks = 0, max_contrib = 0, max_helem_padded = 0;  // padded list lengths of the largest block
  int64_t n_tasks = 0, n_contrib = 0, n_helem_total = 0;
  size_t bytes = 0;
  RowBlock* blocks = nullptr;
  int32_t* lnodes = nullptr;      // per block: owned nodes, then the other nodes of its halo elements
  int32_t* helem_id = nullptr;    // original element id of every halo element
  uint8_t* helem_type = nullptr;
  uint16_t* helem_ln = nullptr;   // [halo element][8] local node ids (block-task plans of hex meshes)
  RowTask* tasks = nullptr;
  uint16_t* contrib = nullptr;
  // block-task plans: runs (first node, count <= kZeroRunNodes) of the nodes
  // whose elements lie in more than one block, the only nodes whose rows hold
  // entries that several blocks add to (every other row is stored whole)
  int32_t* zero_runs = nullptr;
  int64_t n_zero_runs = 0;
};

// (runs of 4 nodes spread the long runs of consecutive boundary nodes over
// warps: at 128^3 with 64-element blocks the 2.34 GB cleared took 0.48 ms in
// runs of up to 64 nodes, 0.42 ms in runs of up to 4, against 0.54 ms for
// clearing all 4.16 GB of A)
constexpr int kZeroRunNodes = 4;

// Zero the rows of A that the block-task kernels add to (the nodes of
// P.zero_runs) instead of all of A: every other row is written whole by
// stores.  Stream-ordered; A 16-byte aligned.
int zero_block_rows(const RowsPlan& P, const int64_t* row_ptr, double* A, cudaStream_t s);

// host-side lists of one block while a plan is built
struct HostBlock {
  std::vector<int32_t> lnodes;     // rows first (owned nodes), then the other local nodes
  std::vector<int32_t> helem;      // original element ids
  std::vector<uint8_t> htype;
  std::vector<uint16_t> hln;       // [helem][8] local node ids (block-task plans of hex meshes only)
  std::vector<RowTask> tasks;
  std::vector<uint16_t> contrib;
  int n_owned = 0;
};

int upload_plan(std::vector<HostBlock>& blocks, int ndof, int block_nodes, int halo_cap, bool all_hex,
                RowsPlan** out);
int build_rows_plan(fea_mesh* m, int ndof, int block_nodes, int halo_cap, cudaStream_t s, RowsPlan** out);
// Block-task plan (FEA_SCATTER_BLOCK): blocks of at most block_elems elements
// along a Morton curve of the element centroids; every entry touched by a
// block is one task, flagged atomic when elements outside the block add to it.
int build_blocks_plan(fea_mesh* m, int ndof, int block_elems, cudaStream_t s, RowsPlan** out);
// the plan for (ndof, precision), built on first use with a halo cap that lets
// two CTAs share an SM; if a block still does not fit, the node cap is halved
int ensure_rows_plan(fea_mesh* m, int ndof, int precision, cudaStream_t s, RowsPlan** out);
void drop_rows_plans(fea_mesh* m);
void free_rows_plan(RowsPlan* P);
RowsLayout rows_layout(const RowsPlan& P, bool stage, int rec_floats = kRowsRecSmem, bool node_data = true);
int assemble_rows(const fea_operator* op, fea_mesh* m, const int64_t* row_ptr, double* A, double* b,
                  cudaStream_t s, int* launched);
// the block-task plan of a mesh, built on first use
int ensure_blocks_plan(fea_mesh* m, int ndof, cudaStream_t s, RowsPlan** out);
// launch the task kernel of a plan (ROWS or BLOCK) on precomputed geometry records
// Block-task plans of hex meshes in FEA_FP32_INTEGRATE compute the geometry
// records inside the task kernel (every element belongs to one block).
bool fused_geometry(const fea_operator* op, const RowsPlan& RP);
// mesh: non-null enables the fused geometry where fused_geometry() holds
int launch_task_kernel(const fea_operator* op, const RowsPlan& RP, const void* records, const int64_t* row_ptr,
                       double* A, double* b, DevStatus* st, cudaStream_t s, const fea_mesh* mesh);

}  // namespace fea
