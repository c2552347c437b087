// rows_kernel.cu -- the CTA kernel of the owner-computes row assembly.
//
// One CTA owns one node block of the plan built in rows.cu.  Its task list
// (one task per entry block (i, j) of its rows), the element-contribution
// codes and the ids of its halo elements arrive by TMA bulk copy into shared
// memory; the per-element data -- scaled gradients g^_a(q), weights and k(x_q)
// -- come from the geometry records written by the geometry pass (read through
// L1, so the records of halo elements shared by neighbouring blocks are
// fetched from L2 once per block rather than recomputed).
//
// Task (i, j): for each contributing element e (node i at local a, j at b)
//   M_e = sum_q g^_a(q) (x) g^_b(q),   K_e = lam M_e + mu M_e^T + mu tr(M_e) I
// (diffusion: K_e = sum_q k(x_q) g^_a . g^_b); the K_e are summed in FP64
// (FP32_INTEGRATE: each FP32 K_e widened exactly) and written to row i --
// and, transposed, to row j when j belongs to the same block.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <type_traits>

#include "element.cuh"
#include "fea_internal.cuh"
#include "geometry.cuh"
#include "rows.cuh"
#include "tma.cuh"

namespace fea {

struct RowsArgs {
  const RowBlock* blocks;
  const int32_t* lnodes;
  const uint8_t* helem_type;
  const RowTask* tasks;
  const uint16_t* contrib;
  const int32_t* helem_id;
  const int64_t* row_ptr;
  const void* rec;          // geometry records (float or double, kRecStride values per element)
  double* A;
  double* b;
  DevStatus* st;
  int64_t n_blocks;
  int tet_nq;               // quadrature points of tet4 (1 or 4)
  RowsLayout L;
  double lam, mu, src, f[3];
  float lamf, muf;                // lam and mu rounded to FP32 on the host (FP32 tiles)
  float Ntab[kNumRules][8][8];    // N_a(q) per rule slot, for the right-hand side
  double Ntab64[kNumRules][8][8];
  // fused geometry (block-task plan, hex8, FP32-integrate): the CTA computes
  // the records of its own elements from the mesh instead of reading them
  const double* coords;
  const int64_t* conn_off;
  const int32_t* conn;
  const uint16_t* helem_ln;       // [halo element][8] block-local node of each corner (pipelined kernel)
  double k0, k2;
  int diffusion;
  RefRule hex;
};

__device__ __forceinline__ int rule_slot_of(int type, int tet_nq) {
  return type == FEA_TET4 ? (tet_nq == 1 ? kRuleTet1 : kRuleTet4)
                          : type == FEA_PYR5 ? kRulePyr8 : type == FEA_PRISM6 ? kRulePrism6 : kRuleHex8;
}

// accumulator of one entry: FP64 sums.  FP32-integrate contributions are
// widened exactly (integer instructions) and added in FP64, so the entry is
// the FP64 sum of the FP32 element contributions, rounded at every add like
// the atomic scatter's.  (An error-free FP32 pair (TwoSum) with one final
// rounding measured slower on GB300: its renormalisation and integer FP64
// assembly per entry cost more than one FP64 add per contribution.)
template <int PREC>
struct Acc;
template <>
struct Acc<FEA_FP64> {
  double v = 0.0;
  __device__ __forceinline__ void set(double x) { v = x; }
  __device__ __forceinline__ void add(double x) { v += x; }
  __device__ __forceinline__ double value() const { return v; }
};
template <>
struct Acc<FEA_FP32_INTEGRATE> {
  double v = 0.0;
  __device__ __forceinline__ void set(float x) { v = f32_to_f64_exact(x); }
  __device__ __forceinline__ void add(float x) { v += f32_to_f64_exact(x); }
  __device__ __forceinline__ double value() const { return v; }
};

static_assert(RecCopied::q * 8 == kRecW && RecCopied::w == kRecW && RecCopied::k == kRecK,
              "staged copies keep the geometry pass's record layout");
// (pipe records are written and read with scalar accesses only, never bulk
// copied, so their stride need not be a 16-byte multiple)
static_assert(RecPipe::q >= 24 && RecPipe::q * 8 <= RecPipe::w && RecPipe::w + 8 <= RecPipe::k &&
                  RecPipe::k + 8 <= RecPipe::stride,
              "pipe records hold 8 x 8 x 3 gradients, 8 weights and 8 conductivities");

// element data: staged in shared memory, or read through L1
template <bool STAGE, typename R>
__device__ __forceinline__ R ld_rec(const R* p) {
  if constexpr (STAGE)
    return *p;
  else
    return __ldg(p);
}

// HEX: every element is a hex8 with 8 points (compile-time loop bounds).
// FP32 record (layout L) of point p (= the thread's lane in its group of 8)
// of a hex element whose corner p has coordinates v, from the FP64 modal
// Jacobian: every lane of the warp calls it.  *id (the element's original id)
// is read only to report an inverted element.
template <class L>
__device__ __forceinline__ void hex_record(const RowsArgs& P, bool valid, const int32_t* id, double v[3],
                                           float* rec) {
  const int p = threadIdx.x & 7;
  hex8_modal(v);
  double c[8][3];
  const int base = threadIdx.x & 24;
#pragma unroll
  for (int k = 0; k < 8; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i) c[k][i] = __shfl_sync(0xffffffffu, v[i], base | k);
  double J[3][3];
  hex8_jacobian_pairs<false>(c, p, J);  // every lane (it exchanges columns)
  if (!valid) return;
  double C[3][3];
  cofactors(J, C);
  const double det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
  if (!(det > 0.0)) {
    latch_error(P.st, FEA_ERR_INVERTED_ELEMENT, (unsigned long long)*id);
    return;
  }
  // J' = 8 J: det J = det'/512, J^{-T} = 8 C'/det'
  float Cf[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Cf[i][j] = f64_to_f32_rn(C[i][j]);
  const float detf = f64_to_f32_rn(det);
  const float wdf = P.hex.wf[p] * detf * (1.0f / 512.0f);
  const float sc = sqrtf(wdf) * 8.0f / detf;
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i)
      rec[p * L::q + 3 * a + i] =
          (P.hex.dNf[p][a][0] * Cf[i][0] + P.hex.dNf[p][a][1] * Cf[i][1] + P.hex.dNf[p][a][2] * Cf[i][2]) * sc;
  rec[L::w + p] = wdf;
  if (P.diffusion) {
    const float x = f64_to_f32_rn(hex8_modal_x(c, p));
    rec[L::k + p] = f64_to_f32_rn(P.k0) + f64_to_f32_rn(P.k2) * x * x;
  }
}

// the same, with corner p's coordinates read from the mesh
template <class L>
__device__ __forceinline__ void fused_hex_record(const RowsArgs& P, bool valid, const int32_t* id, float* rec) {
  double v[3] = {0.0, 0.0, 0.0};
  if (valid) {
    const int64_t node = P.conn[P.conn_off[*id] + hex8_corner_node(threadIdx.x & 7)];
#pragma unroll
    for (int i = 0; i < 3; ++i) v[i] = P.coords[3 * node + i];
  }
  hex_record<L>(P, valid, id, v, rec);
}

// an operator parameter in the tile precision (FP32 values rounded on the host)
template <typename R>
__device__ __forceinline__ R tile_param(double d, float f);
template <>
__device__ __forceinline__ double tile_param<double>(double d, float) {
  return d;
}
template <>
__device__ __forceinline__ float tile_param<float>(double, float f) {
  return f;
}

// three consecutive values of A at p = A + e: one 16-byte and one 8-byte
// store (A is 16-byte aligned, so p is when e is even) instead of three, and
// fewer sectors to request from L2
__device__ __forceinline__ void store3(double* p, int64_t e, double a0, double a1, double a2) {
  if ((e & 1) == 0) {
    *reinterpret_cast<double2*>(p) = make_double2(a0, a1);
    p[2] = a2;
  } else {
    p[0] = a0;
    *reinterpret_cast<double2*>(p + 1) = make_double2(a1, a2);
  }
}

// One entry-block task t of a block: its element contributions summed in
// registers, the entry block stored (or added, at block boundaries) to row i
// and, transposed, to row j; the right-hand side of node i with the
// diagonal task.  Records staged in shared memory when STAGE, in layout L,
// else read from `rec`, whose records have L's offsets and kRecStride values
// each.
template <int OP, int PREC, bool HEX, bool STAGE, class L>
__device__ __forceinline__ void run_task(const RowsArgs& P, const RowBlock& H,
                                         const typename std::conditional<PREC == FEA_FP64, double, float>::type* s_recs,
                                         const int64_t* s_rs, const RowTask* s_tasks, const uint16_t* s_contrib,
                                         const int32_t* s_hid, const int32_t* gnode, int t) {
  using R = typename std::conditional<PREC == FEA_FP64, double, float>::type;
  constexpr int D = OP == FEA_OP_DIFFUSION ? 1 : 3;
  const R* rec = reinterpret_cast<const R*>(P.rec);
  const R lam = tile_param<R>(P.lam, P.lamf), mu = tile_param<R>(P.mu, P.muf);
  const RowTask T = s_tasks[t];
  const bool diag = T.flags & kTaskDiag;
  Acc<PREC> acc[D][D];
  Acc<PREC> bsum;   // sum over the contributions of w det J N_a (b_i = f times it)
#pragma unroll 1
  for (int c = 0; c < T.nc; ++c) {
    const int code = s_contrib[T.coff + c];
    const int h = code >> 6, a = (code >> 3) & 7, bn = code & 7;
    const int type = HEX ? (int)FEA_HEX8 : (int)__ldg(P.helem_type + H.helem_off + h);
    const int nq = HEX ? 8 : (type == FEA_TET4 ? P.tet_nq : type == FEA_PRISM6 ? 6 : 8);
    const R* re = STAGE ? s_recs + (size_t)h * L::stride : rec + (int64_t)s_hid[h] * kRecStride;
    const R* ga = re + 3 * a;
    const R* gb = re + 3 * bn;
    R K[D][D];
    if constexpr (OP == FEA_OP_DIFFUSION) {
      R s = R(0);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (!HEX && q >= nq) break;
        const R x0 = ld_rec<STAGE>(ga + L::q * q), x1 = ld_rec<STAGE>(ga + L::q * q + 1),
                x2 = ld_rec<STAGE>(ga + L::q * q + 2);
        const R y0 = ld_rec<STAGE>(gb + L::q * q), y1 = ld_rec<STAGE>(gb + L::q * q + 1),
                y2 = ld_rec<STAGE>(gb + L::q * q + 2);
        s += ld_rec<STAGE>(re + L::k + q) * (x0 * y0 + x1 * y1 + x2 * y2);
      }
      K[0][0] = s;
    } else {
      R M[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (!HEX && q >= nq) break;
        const R x0 = ld_rec<STAGE>(ga + L::q * q), x1 = ld_rec<STAGE>(ga + L::q * q + 1),
                x2 = ld_rec<STAGE>(ga + L::q * q + 2);
        const R y0 = ld_rec<STAGE>(gb + L::q * q), y1 = ld_rec<STAGE>(gb + L::q * q + 1),
                y2 = ld_rec<STAGE>(gb + L::q * q + 2);
        M[0][0] += x0 * y0; M[0][1] += x0 * y1; M[0][2] += x0 * y2;
        M[1][0] += x1 * y0; M[1][1] += x1 * y1; M[1][2] += x1 * y2;
        M[2][0] += x2 * y0; M[2][1] += x2 * y1; M[2][2] += x2 * y2;
      }
      const R tr = mu * (M[0][0] + M[1][1] + M[2][2]);
#pragma unroll
      for (int c1 = 0; c1 < 3; ++c1)
#pragma unroll
        for (int c2 = 0; c2 < 3; ++c2) K[c1][c2] = lam * M[c1][c2] + mu * M[c2][c1] + (c1 == c2 ? tr : R(0));
    }
    if (c == 0) {
#pragma unroll
      for (int c1 = 0; c1 < D; ++c1)
#pragma unroll
        for (int c2 = 0; c2 < D; ++c2) acc[c1][c2].set(K[c1][c2]);
    } else {
#pragma unroll
      for (int c1 = 0; c1 < D; ++c1)
#pragma unroll
        for (int c2 = 0; c2 < D; ++c2) acc[c1][c2].add(K[c1][c2]);
    }
    if (diag) {
      const int slot = HEX ? (int)kRuleHex8 : rule_slot_of(type, P.tet_nq);
      R rb = R(0);
      for (int q = 0; q < nq; ++q) {
        R Nqa;
        if constexpr (PREC == FEA_FP64)
          Nqa = P.Ntab64[slot][q][a];
        else
          Nqa = P.Ntab[slot][q][a];
        rb += ld_rec<STAGE>(re + L::w + q) * Nqa;
      }
      if (c == 0)
        bsum.set(rb);
      else
        bsum.add(rb);
    }
  }
  // the entry block, rounded once, to row i and transposed to row j
  double v[D][D];
#pragma unroll
  for (int c1 = 0; c1 < D; ++c1)
#pragma unroll
    for (int c2 = 0; c2 < D; ++c2) v[c1][c2] = acc[c1][c2].value();
  // complete entries are stored; block-boundary entries (block-task plan)
  // are added to A with FP64 atomics
  const bool at = T.flags & kTaskAtomicA;
#pragma unroll
  for (int c1 = 0; c1 < D; ++c1) {
    const int64_t base = s_rs[D * T.li + c1] + (int64_t)D * T.k;
    if (at) {
#pragma unroll
      for (int c2 = 0; c2 < D; ++c2) red_add(P.A + base + c2, v[c1][c2]);
    } else if constexpr (D == 3) {
      store3(P.A + base, base, v[c1][0], v[c1][1], v[c1][2]);
    } else {
      P.A[base] = v[0][0];
    }
  }
  if (T.flags & kTaskTranspose) {
#pragma unroll
    for (int c2 = 0; c2 < D; ++c2) {
      const int64_t base = s_rs[D * T.lj + c2] + (int64_t)D * T.kt;
      if (at) {
#pragma unroll
        for (int c1 = 0; c1 < D; ++c1) red_add(P.A + base + c1, v[c1][c2]);
      } else if constexpr (D == 3) {
        store3(P.A + base, base, v[0][c2], v[1][c2], v[2][c2]);
      } else {
        P.A[base] = v[0][0];
      }
    }
  }
  if (diag) {
    // the source is constant over the mesh: b_i = f (sum of the element
    // integrals of N_a), one FP64 product per component
    const int64_t gi = gnode[T.li];
    const double beta = bsum.value();
#pragma unroll
    for (int c1 = 0; c1 < D; ++c1) {
      const double bv = beta * (OP == FEA_OP_DIFFUSION ? P.src : P.f[c1]);
      if (T.flags & kTaskAtomicB)
        red_add(P.b + D * gi + c1, bv);
      else
        P.b[D * gi + c1] = bv;
    }
  }
}

// the first of the next 32 tasks of the block, for the whole warp (every
// lane calls it)
__device__ __forceinline__ int grab_tasks(int* s_next) {
  int t0 = 0;
  if ((threadIdx.x & 31) == 0) t0 = atomicAdd(s_next, 32);
  return __shfl_sync(0xffffffffu, t0, 0);
}

// the first of the next 4 elements of the block, for the whole warp
__device__ __forceinline__ int grab_elements(int* s_enext) {
  int e0 = 0;
  if ((threadIdx.x & 31) == 0) e0 = atomicAdd(s_enext, 4);
  return __shfl_sync(0xffffffffu, e0, 0);
}

// The entry-block tasks of one block, 32 consecutive tasks per warp.  The
// tasks are sorted by contribution count, largest first.  With s_next (a
// shared counter, zero at the start of the block) the warps take batches as
// they finish, so the largest go first and no warp is left holding all of
// them; without it the warp of threads tid..tid+31 takes batches tid,
// tid + nthreads, ... (tid a multiple of 32 at the warp's first lane,
// nthreads a multiple of 32).  Which warp runs a task does not change what it
// computes.
template <int OP, int PREC, bool HEX, bool STAGE, class L = RecCopied>
__device__ __forceinline__ void run_tasks(const RowsArgs& P, const RowBlock& H,
                                          const typename std::conditional<PREC == FEA_FP64, double, float>::type* s_recs,
                                          const int64_t* s_rs, const RowTask* s_tasks, const uint16_t* s_contrib,
                                          const int32_t* s_hid, const int32_t* gnode, int tid, int nthreads,
                                          int* s_next = nullptr) {
  for (int t0 = s_next ? grab_tasks(s_next) : (tid & ~31); t0 < H.n_tasks;
       t0 = s_next ? grab_tasks(s_next) : t0 + nthreads) {
    const int t = t0 + (tid & 31);
    if (t < H.n_tasks) run_task<OP, PREC, HEX, STAGE, L>(P, H, s_recs, s_rs, s_tasks, s_contrib, s_hid, gnode, t);
  }
}

// STAGE: the halo elements' records are bulk-copied into shared memory (FP32).
// GEO (with STAGE and HEX): the CTA computes them there from the mesh instead.
template <int OP, int PREC, bool HEX, bool STAGE, bool GEO = false>
__global__ void __launch_bounds__(256, 2) k_rows_assemble(const __grid_constant__ RowsArgs P) {
  static_assert(!GEO || (STAGE && HEX), "fused geometry computes staged hex records");
  using R = typename std::conditional<PREC == FEA_FP64, double, float>::type;
  constexpr int D = OP == FEA_OP_DIFFUSION ? 1 : 3;
  static_assert(!STAGE || PREC != FEA_FP64, "records are staged in FP32 only");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* s_recs = reinterpret_cast<R*>(smem_raw + P.L.recs);
  int64_t* s_rs = reinterpret_cast<int64_t*>(smem_raw + P.L.rs);
  RowTask* s_tasks = reinterpret_cast<RowTask*>(smem_raw + P.L.tasks);
  uint16_t* s_contrib = reinterpret_cast<uint16_t*>(smem_raw + P.L.contrib);
  int32_t* s_hid = reinterpret_cast<int32_t*>(smem_raw + P.L.hid);
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem_raw + P.L.bar);
  const R* rec = reinterpret_cast<const R*>(P.rec);
  if (threadIdx.x == 0) mbar_init(s_bar);
  __shared__ int s_next;  // the block's next batch of tasks
  __syncthreads();
  uint32_t parity = 0;
  for (int64_t blk = blockIdx.x; blk < P.n_blocks; blk += gridDim.x, parity ^= 1u) {
    const RowBlock H = P.blocks[blk];
    if (threadIdx.x < 32) {
      const uint32_t rec_bytes = (STAGE && !GEO) ? (uint32_t)(4 * kRecStride) * H.n_helem : 0u;
      if (threadIdx.x == 0) {
        s_next = 0;  // read after the barrier below
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // order earlier reads of the buffers
        mbar_expect_tx(s_bar, H.task_bytes + H.contrib_bytes + H.helem_bytes + rec_bytes);
        if (H.task_bytes) bulk_copy_g2s(s_tasks, P.tasks + H.task_off, H.task_bytes, s_bar);
        if (H.contrib_bytes) bulk_copy_g2s(s_contrib, P.contrib + H.contrib_off, H.contrib_bytes, s_bar);
        if (H.helem_bytes) bulk_copy_g2s(s_hid, P.helem_id + H.helem_off, H.helem_bytes, s_bar);
      }
      if constexpr (STAGE && !GEO) {
        // one 832-byte record per halo element (16-byte aligned at both ends)
        __syncwarp();
        for (int h = threadIdx.x; h < H.n_helem; h += 32) {
          const int64_t id = P.helem_id[H.helem_off + h];
          bulk_copy_g2s(s_recs + (size_t)h * kRowsRecSmem, rec + id * kRecStride, 4u * kRecStride, s_bar);
        }
      }
    }
    const int32_t* lnodes = P.lnodes + H.lnode_off;
    for (int t = threadIdx.x; t < H.n_owned * D; t += blockDim.x)
      s_rs[t] = P.row_ptr[(int64_t)D * lnodes[t / D] + t % D];
    if constexpr (GEO) {
      // the block's elements, 32 at a time (8 threads each), while the task
      // lists are still in flight
      for (int h0 = 0; h0 < H.n_helem; h0 += 32) {
        const int h = h0 + (threadIdx.x >> 3);
        const bool valid = h < H.n_helem;
        fused_hex_record<RecCopied>(P, valid, P.helem_id + H.helem_off + (valid ? h : 0),
                                    reinterpret_cast<float*>(s_recs) + (size_t)(valid ? h : 0) * kRowsRecSmem);
      }
    }
    const bool landed = mbar_wait_bounded(s_bar, parity);
    if (__syncthreads_or(!landed)) {
      // the copy did not land within the bound: report, wait a last bounded
      // while for the copy in flight, and leave without touching A
      if (threadIdx.x == 0) latch_error(P.st, FEA_ERR_TIMEOUT, (unsigned long long)blk);
      mbar_wait_bounded(s_bar, parity);
      return;
    }
    run_tasks<OP, PREC, HEX, STAGE>(P, H, s_recs, s_rs, s_tasks, s_contrib, s_hid, lnodes, threadIdx.x, blockDim.x,
                                    &s_next);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Block-task plans of hex meshes in FP32-integrate, pipelined: one persistent
// CTA per SM works through its blocks blk = blockIdx.x + i gridDim.x.  Two
// shared-memory stages hold a block's task lists and records; three node
// buffers hold its nodes' row starts, ids and coordinates and its elements'
// corner lists.
//  * Warps 0..PW-1 (producers) compute the FP64-geometry records of block i
//    from node buffer i % 3 into stage i & 1, 4 elements per warp at a time
//    from a per-stage counter; a warp that finds none left arrives on full[s]
//    and goes on to block i + 1, so no producer waits for another.
//  * Warp 0 also leads: once the consumers release stage i & 1 (block
//    i - 2) it starts the TMA bulk copies of block i's task lists into it and
//    arrives on ready[i % 3], which lets the producers start; then, before its
//    own share of block i, it gathers block i + 1's node data into node buffer
//    (i + 1) % 3 (last read by block i - 2).  The gather is off the chain
//    from one block's release to the next one's records.
//  * Warps PW..15 (consumers) run the tasks of the block whose stage is full,
//    32 at a time from a per-stage counter (the tasks are sorted largest
//    first; with a fixed share the first consumer warp would hold the largest
//    of every round, and the stage is released only when its slowest
//    consumer is done).
// mbarriers hand the buffers over: ready[b] (32 lead arrivals), full[s] (1
// arrival with the copy bytes + 32 PW producer arrivals) and empty[s]
// (32 (16 - PW) consumer arrivals).  Every wait is bounded; a timeout latches
// FEA_ERR_TIMEOUT and every role leaves its loop at its next look at the
// shared failure flag (no role waits at a named barrier); the copies in
// flight are waited for before exit.  The producer/consumer split is a
// template parameter, chosen per mesh (fea_mesh_set_pipe_split, or the
// autotuner).
// ---------------------------------------------------------------------------
constexpr int kPipeThreads = 512;
constexpr int kGatherPerLane = 4;  // node loads in flight per gathering lane

// Shared-memory layout of the pipelined kernel (byte offsets from the start
// of dynamic shared memory, or within a node buffer)
struct PipeLayout {
  uint32_t stage_bytes;                    // one stage (rows_layout without node data, 128-byte multiple)
  uint32_t node_off;                       // node buffer 0 (buffer b at node_off + b node_bytes)
  uint32_t node_bytes;                     // one node buffer:
  uint32_t x_rel, ln_rel, rs_rel, gi_rel;  // coordinates, corner lists, row starts, node ids
  uint32_t total;
};

__device__ __forceinline__ void pipe_fail(const RowsArgs& P, int* s_fail, int64_t blk) {
  if (atomicExch(s_fail, 1) == 0) latch_error(P.st, FEA_ERR_TIMEOUT, (unsigned long long)blk);
}

// block blk's node data into node buffer nb, by one warp (lane = 0..31):
// kGatherPerLane node ids per lane in flight, then their row starts and
// coordinates, then the elements' corner lists (8 x 16 bits each)
template <int D>
__device__ __forceinline__ void pipe_gather(const RowsArgs& P, const PipeLayout& PL, int64_t blk,
                                            unsigned char* nb, int lane) {
  const RowBlock H = P.blocks[blk];
  double* n_x = reinterpret_cast<double*>(nb + PL.x_rel);
  int64_t* n_rs = reinterpret_cast<int64_t*>(nb + PL.rs_rel);
  int32_t* n_gi = reinterpret_cast<int32_t*>(nb + PL.gi_rel);
  const int32_t* lnodes = P.lnodes + H.lnode_off;
  for (int t0 = 0; t0 < H.n_local; t0 += 32 * kGatherPerLane) {
    int32_t node[kGatherPerLane];
#pragma unroll
    for (int k = 0; k < kGatherPerLane; ++k) {
      const int t = t0 + 32 * k + lane;
      node[k] = t < H.n_local ? lnodes[t] : -1;
    }
    int64_t rs[kGatherPerLane][D];
    double x[kGatherPerLane][3];
#pragma unroll
    for (int k = 0; k < kGatherPerLane; ++k) {
      const int64_t nd = node[k] < 0 ? 0 : node[k];
#pragma unroll
      for (int c = 0; c < D; ++c) rs[k][c] = node[k] < 0 ? 0 : P.row_ptr[(int64_t)D * nd + c];
#pragma unroll
      for (int c = 0; c < 3; ++c) x[k][c] = node[k] < 0 ? 0.0 : P.coords[3 * nd + c];
    }
#pragma unroll
    for (int k = 0; k < kGatherPerLane; ++k) {
      const int t = t0 + 32 * k + lane;
      if (t < H.n_local) {
        if (t < H.n_owned) {
          n_gi[t] = node[k];
#pragma unroll
          for (int c = 0; c < D; ++c) n_rs[D * t + c] = rs[k][c];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) n_x[3 * t + c] = x[k][c];
      }
    }
  }
  uint4* n_ln = reinterpret_cast<uint4*>(nb + PL.ln_rel);
  for (int t = lane; t < H.n_helem; t += 32) n_ln[t] = reinterpret_cast<const uint4*>(P.helem_ln)[H.helem_off + t];
}

template <int OP, int PW>
__global__ void __launch_bounds__(kPipeThreads, 1)
    k_block_pipe(const __grid_constant__ RowsArgs P, const PipeLayout PL) {
  constexpr int kProducers = 32 * PW;
  constexpr int kConsumers = kPipeThreads - kProducers;
  constexpr int D = OP == FEA_OP_DIFFUSION ? 1 : 3;
  extern __shared__ __align__(128) unsigned char pipe_raw[];
  uint64_t* full = reinterpret_cast<uint64_t*>(pipe_raw + 2 * PL.stage_bytes);
  uint64_t* empty = full + 2;
  uint64_t* ready = full + 4;  // three
  __shared__ int s_issued[2];
  __shared__ int s_next[2];   // each stage's next batch of tasks
  __shared__ int s_enext[2];  // each stage's next 4 elements
  __shared__ int s_fail;
  if (threadIdx.x == 0) {
    for (int k = 0; k < 2; ++k) {
      mbar_init_count(&full[k], kProducers + 1);
      mbar_init_count(&empty[k], kConsumers);
      s_issued[k] = 0;
    }
    for (int k = 0; k < 3; ++k) mbar_init_count(&ready[k], 32);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5;
  auto node_buf = [&](int i) { return pipe_raw + PL.node_off + (size_t)(i % 3) * PL.node_bytes; };
  int i = 0;
  if (warp < PW) {
    // the producers; warp 0 leads
    const bool lead = warp == 0;
    const int lane = threadIdx.x & 31;
    if (lead && blockIdx.x < P.n_blocks) pipe_gather<D>(P, PL, blockIdx.x, node_buf(0), lane);
    for (int64_t blk = blockIdx.x; blk < P.n_blocks; blk += gridDim.x, ++i) {
      const int s = i & 1;
      if (*((volatile int*)&s_fail)) break;
      if (lead) {
        // the consumers have released this stage (block i - 2), and with it
        // the producers are done with its records and counter
        if (i >= 2 && !mbar_wait_bounded(&empty[s], ((uint32_t)(i >> 1) & 1u) ^ 1u)) {
          if (lane == 0) pipe_fail(P, &s_fail, blk);
          break;
        }
        if (lane == 0) {
          const RowBlock H = P.blocks[blk];
          unsigned char* base = pipe_raw + (size_t)s * PL.stage_bytes;
          s_next[s] = 0;   // published to the consumers through full[s]
          s_enext[s] = 0;  // and to the producers through ready[i % 3]
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // earlier reads of the stage
          mbar_expect_tx(&full[s], H.task_bytes + H.contrib_bytes + H.helem_bytes);
          if (H.task_bytes) bulk_copy_g2s(base + P.L.tasks, P.tasks + H.task_off, H.task_bytes, &full[s]);
          if (H.contrib_bytes)
            bulk_copy_g2s(base + P.L.contrib, P.contrib + H.contrib_off, H.contrib_bytes, &full[s]);
          if (H.helem_bytes) bulk_copy_g2s(base + P.L.hid, P.helem_id + H.helem_off, H.helem_bytes, &full[s]);
          ++s_issued[s];
        }
        mbar_arrive(&ready[i % 3]);
        // the next block's node data (its buffer was last read by block i - 2)
        if (blk + gridDim.x < P.n_blocks) pipe_gather<D>(P, PL, blk + gridDim.x, node_buf(i + 1), lane);
      }
      if (!mbar_wait_bounded(&ready[i % 3], (uint32_t)(i / 3) & 1u)) {
        pipe_fail(P, &s_fail, blk);
        break;
      }
      const int n_helem = P.blocks[blk].n_helem;
      const int64_t helem_off = P.blocks[blk].helem_off;
      float* s_recs = reinterpret_cast<float*>(pipe_raw + (size_t)s * PL.stage_bytes + P.L.recs);
      const unsigned char* nb = node_buf(i);
      const double* n_x = reinterpret_cast<const double*>(nb + PL.x_rel);
      const uint16_t* n_ln = reinterpret_cast<const uint16_t*>(nb + PL.ln_rel);
      // a warp holds 4 elements (8 lanes each) and takes the next 4 when done
      for (int h0 = grab_elements(&s_enext[s]); h0 < n_helem; h0 = grab_elements(&s_enext[s])) {
        const int h = h0 + (lane >> 3);
        const bool valid = h < n_helem;
        double v[3] = {0.0, 0.0, 0.0};
        if (valid) {
          const int ln = n_ln[8 * h + hex8_corner_node(threadIdx.x & 7)];
#pragma unroll
          for (int c = 0; c < 3; ++c) v[c] = n_x[3 * ln + c];
        }
        hex_record<RecPipe>(P, valid, P.helem_id + helem_off + (valid ? h : 0), v,
                            s_recs + (size_t)(valid ? h : 0) * RecPipe::stride);
      }
      mbar_arrive(&full[s]);
    }
  } else {
    // the consumers
    for (int64_t blk = blockIdx.x; blk < P.n_blocks; blk += gridDim.x, ++i) {
      const int s = i & 1;
      if (*((volatile int*)&s_fail)) break;
      if (!mbar_wait_bounded(&full[s], (uint32_t)(i >> 1) & 1u)) {
        pipe_fail(P, &s_fail, blk);
        break;
      }
      const RowBlock H = P.blocks[blk];
      const unsigned char* base = pipe_raw + (size_t)s * PL.stage_bytes;
      const unsigned char* nb = node_buf(i);
      run_tasks<OP, FEA_FP32_INTEGRATE, true, true, RecPipe>(
          P, H, reinterpret_cast<const float*>(base + P.L.recs), reinterpret_cast<const int64_t*>(nb + PL.rs_rel),
          reinterpret_cast<const RowTask*>(base + P.L.tasks), reinterpret_cast<const uint16_t*>(base + P.L.contrib),
          reinterpret_cast<const int32_t*>(base + P.L.hid), reinterpret_cast<const int32_t*>(nb + PL.gi_rel),
          (int)threadIdx.x - kProducers, kConsumers, &s_next[s]);
      mbar_arrive(&empty[s]);
    }
  }
  __syncthreads();
  // after a timeout: let the bulk copies still in flight land before exit
  if (threadIdx.x == 0 && s_fail)
    for (int k = 0; k < 2; ++k)
      if (s_issued[k] > 0) mbar_wait_bounded(&full[k], (uint32_t)((s_issued[k] - 1) & 1));
}

int assemble_rows(const fea_operator* op, fea_mesh* m, const int64_t* row_ptr, double* A, double* b,
                  cudaStream_t s, int* launched) {
  const int D = op->kind == FEA_OP_DIFFUSION ? 1 : 3;
  RowsPlan* plan = nullptr;
  int rc = ensure_rows_plan(m, D, op->precision, s, &plan);
  if (rc) return rc;
  void* records = nullptr;
  int geo_launches = 0;
  rc = geometry_pass(op, m, s, &records, &geo_launches);
  if (rc) return rc;
  rc = launch_task_kernel(op, *plan, records, row_ptr, A, b, m->status, s, nullptr);
  if (rc == FEA_OK) *launched = geo_launches + 1;
  return rc;
}

// 32 zero bytes at a 32-byte aligned address
__device__ __forceinline__ void zero32(double* p) {
  asm volatile("st.global.v4.f64 [%0], {%1, %1, %1, %1};" ::"l"(__cvta_generic_to_global(p)), "d"(0.0) : "memory");
}

// A warp per run of nodes: their rows of A, [row_ptr[D first], row_ptr[D
// (first + count)]), are contiguous; zeroed with 32-byte stores from the
// first 32-byte boundary on, single values before it and after the last one.
__global__ void __launch_bounds__(256) k_zero_rows(const int32_t* runs, int64_t n_runs, const int64_t* row_ptr,
                                                   int D, double* A) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n_runs; r += nwarps) {
    const int64_t first = runs[2 * r], count = runs[2 * r + 1];
    int64_t lo = row_ptr[(int64_t)D * first];
    const int64_t hi = row_ptr[(int64_t)D * (first + count)];
    int64_t head = (int64_t)(((32u - ((uint32_t)(uintptr_t)(A + lo) & 31u)) & 31u) >> 3);
    if (head > hi - lo) head = hi - lo;
    if (lane < head) A[lo + lane] = 0.0;
    lo += head;
    const int64_t quads = (hi - lo) >> 2;
    for (int64_t k = lane; k < quads; k += 32) zero32(A + lo + 4 * k);
    const int64_t rest = (hi - lo) & 3;
    if (lane < rest) A[lo + 4 * quads + lane] = 0.0;
  }
}

int zero_block_rows(const RowsPlan& P, const int64_t* row_ptr, double* A, cudaStream_t s) {
  if (P.n_zero_runs == 0) return FEA_OK;
  const int64_t ctas = std::min<int64_t>((P.n_zero_runs + 7) / 8, 152 * 32);
  k_zero_rows<<<(unsigned)ctas, 256, 0, s>>>(P.zero_runs, P.n_zero_runs, row_ptr, P.ndof, A);
  FEA_CUDA(cudaGetLastError());
  return FEA_OK;
}

bool fused_geometry(const fea_operator* op, const RowsPlan& RP) {
  return op->precision == FEA_FP32_INTEGRATE && RP.all_hex;
}

int launch_task_kernel(const fea_operator* op, const RowsPlan& RP, const void* records, const int64_t* row_ptr,
                       double* A, double* b, DevStatus* st, cudaStream_t s, const fea_mesh* m) {
  int rc = FEA_OK;
  RowsArgs P;
  std::memset(&P, 0, sizeof(P));
  P.blocks = RP.blocks;
  P.lnodes = RP.lnodes;
  P.helem_type = RP.helem_type;
  P.tasks = RP.tasks;
  P.contrib = RP.contrib;
  P.helem_id = RP.helem_id;
  P.row_ptr = row_ptr;
  P.rec = records;
  P.A = A;
  P.b = b;
  P.st = st;
  P.n_blocks = RP.n_blocks;
  P.tet_nq = op->tet_rule ? 4 : 1;
  const bool stage = op->precision != FEA_FP64;
  P.L = rows_layout(RP, stage);
  const double E = op->young, nu = op->poisson;
  P.lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  P.mu = E / (2.0 * (1.0 + nu));
  P.src = op->source;
  for (int c = 0; c < 3; ++c) P.f[c] = op->body_force[c];
  P.lamf = (float)P.lam;
  P.muf = (float)P.mu;
  for (int k = 0; k < kNumRules; ++k) {
    const RefRule& rr = host_rule(k);
    for (int q = 0; q < 8; ++q)
      for (int a = 0; a < 8; ++a) {
        P.Ntab[k][q][a] = rr.Nf[q][a];
        P.Ntab64[k][q][a] = rr.N[q][a];
      }
  }
  const bool geo = m != nullptr && fused_geometry(op, RP);
  if (geo) {
    P.coords = m->coords;
    P.conn_off = m->conn_off;
    P.conn = m->conn;
    P.k0 = op->k0;
    P.k2 = op->k2;
    P.diffusion = op->kind == FEA_OP_DIFFUSION;
    P.hex = host_rule(kRuleHex8);
    P.helem_ln = RP.helem_ln;
  }
  if (geo) {
    RowsArgs Q = P;
    Q.L = rows_layout(RP, true, RecPipe::stride, false);
    PipeLayout PL;
    PL.stage_bytes = (Q.L.bar + 127u) & ~127u;
    PL.node_off = 2 * PL.stage_bytes + 64;  // after the seven mbarriers
    PL.x_rel = 0;
    PL.ln_rel = (24u * (uint32_t)RP.max_local + 15u) & ~15u;
    PL.rs_rel = PL.ln_rel + 16u * (uint32_t)RP.max_helem;
    PL.gi_rel = PL.rs_rel + 8u * (uint32_t)RP.ndof * (uint32_t)RP.max_owned;
    PL.node_bytes = (PL.gi_rel + 4u * (uint32_t)RP.max_owned + 15u) & ~15u;
    PL.total = PL.node_off + 3 * PL.node_bytes;
    if (PL.total <= kRowsMaxSmem && RP.helem_ln != nullptr) {
      int dev = 0, sms = 0;
      FEA_CUDA(cudaGetDevice(&dev));
      FEA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
      const unsigned grid = (unsigned)std::min<int64_t>(RP.n_blocks, sms);
      const bool dif = op->kind == FEA_OP_DIFFUSION;
      void (*kern)(const RowsArgs, const PipeLayout) = nullptr;
      switch (m->pipe_producer_warps) {
        case 4: kern = dif ? k_block_pipe<FEA_OP_DIFFUSION, 4> : k_block_pipe<FEA_OP_ELASTICITY, 4>; break;
        case 5: kern = dif ? k_block_pipe<FEA_OP_DIFFUSION, 5> : k_block_pipe<FEA_OP_ELASTICITY, 5>; break;
        case 7: kern = dif ? k_block_pipe<FEA_OP_DIFFUSION, 7> : k_block_pipe<FEA_OP_ELASTICITY, 7>; break;
        case 8: kern = dif ? k_block_pipe<FEA_OP_DIFFUSION, 8> : k_block_pipe<FEA_OP_ELASTICITY, 8>; break;
        default: kern = dif ? k_block_pipe<FEA_OP_DIFFUSION, 6> : k_block_pipe<FEA_OP_ELASTICITY, 6>; break;
      }
      FEA_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PL.total));
      kern<<<grid, kPipeThreads, PL.total, s>>>(Q, PL);
      FEA_CUDA(cudaGetLastError());
      return FEA_OK;
    }
  }
  const size_t smem = P.L.total;
  if (smem > kRowsMaxSmem)
    return fail(FEA_ERR_UNSUPPORTED, "rows: a block needs " + std::to_string(smem) + " bytes of shared memory");
  const unsigned grid = (unsigned)RP.n_blocks;
  auto launch = [&](auto kern) -> int {
    FEA_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, 256, smem, s>>>(P);
    FEA_CUDA(cudaGetLastError());
    return FEA_OK;
  };
  const bool hex = RP.all_hex;
  if (op->kind == FEA_OP_DIFFUSION) {
    if (op->precision == FEA_FP64)
      rc = hex ? launch(k_rows_assemble<FEA_OP_DIFFUSION, FEA_FP64, true, false>)
               : launch(k_rows_assemble<FEA_OP_DIFFUSION, FEA_FP64, false, false>);
    else
      rc = geo   ? launch(k_rows_assemble<FEA_OP_DIFFUSION, FEA_FP32_INTEGRATE, true, true, true>)
           : hex ? launch(k_rows_assemble<FEA_OP_DIFFUSION, FEA_FP32_INTEGRATE, true, true>)
                 : launch(k_rows_assemble<FEA_OP_DIFFUSION, FEA_FP32_INTEGRATE, false, true>);
  } else {
    if (op->precision == FEA_FP64)
      rc = hex ? launch(k_rows_assemble<FEA_OP_ELASTICITY, FEA_FP64, true, false>)
               : launch(k_rows_assemble<FEA_OP_ELASTICITY, FEA_FP64, false, false>);
    else
      rc = geo   ? launch(k_rows_assemble<FEA_OP_ELASTICITY, FEA_FP32_INTEGRATE, true, true, true>)
           : hex ? launch(k_rows_assemble<FEA_OP_ELASTICITY, FEA_FP32_INTEGRATE, true, true>)
                 : launch(k_rows_assemble<FEA_OP_ELASTICITY, FEA_FP32_INTEGRATE, false, true>);
  }
  return rc;
}

}  // namespace fea
