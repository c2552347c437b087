// spmv.cu -- the product of an assembled system with a vector, and its
// partial-row form across element partitions.
//
// Sec. 3.1 of the paper partitions the elements; each subdomain assembles
// the square local matrix of its own elements, so a node on an interface
// carries only the partial rows of the subdomains that hold it.  No exchange
// is needed while assembling; the matrix-vector product that follows sums the
// partial rows of interface nodes:  y = sum_p P_p^T (A_p (P_p x)).  On one
// GPU the subdomains are separate meshes (local node numbering, a local ->
// global node map); fea_spmv computes one subdomain's product and adds it into
// the global y -- interface nodes (held by more than one subdomain) with FP64
// atomics, the others with plain stores.
//
// The product reads A through the mesh's own node graph: the d rows of node i
// are one contiguous span of A (d x d x deg(i) values, rows d i .. d i + d - 1),
// and the column of value (c, k, c') is d col_node[rp_node[i] + k] + c'.  So
// no scalar column array is read: per hex node, 1,944 bytes of A and 108 of
// node columns.
#include <algorithm>

#include "element.cuh"
#include "fea_internal.cuh"

namespace fea {

// On GB300 this product is bound by the FP64 pipe (two DFMA per SM and clock)
// about as tightly as by HBM: per 8-byte value of A, one DFMA takes 1.6 ps of
// the GPU's FP64 rate and its bytes 1.2 ps of the HBM copy rate.  So the
// kernel spends FP64 work on the nnz multiply-adds and almost nothing else:
// two lanes per scalar row, lane `sub`
// taking the values t = sub, sub + 2, ... of the row (neighbouring lanes read
// neighbouring values of A, the other half of each sector is the next
// instruction's L1 hit), one shuffle level to finish the row.  No shared
// memory: the load latency is hidden by resident warps.  (A per-warp TMA
// pipeline through shared memory, and four or eight lanes per row, measured
// slower: their reductions and stage waits cost more than they save.)
constexpr int kSpmvLanes = 2;

template <int D>
__global__ void __launch_bounds__(256, 6) k_spmv_rows(const int64_t* __restrict__ rp_node,
                                                      const int32_t* __restrict__ col_node,
                                                      const int64_t* __restrict__ row_ptr,
                                                      const double* __restrict__ A, const double* __restrict__ x,
                                                      double* __restrict__ y, int64_t n_nodes,
                                                      const int32_t* __restrict__ glob,
                                                      const uint8_t* __restrict__ shared) {
  constexpr int L = kSpmvLanes;
  const int sub = threadIdx.x & (L - 1);
  const int64_t n_rows = D * n_nodes;
  const int64_t stride = ((int64_t)gridDim.x * blockDim.x) / L;
  // all lanes of a warp take the same trip count: the shuffle needs them all
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) / L;
  for (int64_t r0 = warp0; r0 < n_rows; r0 += stride) {
    const int64_t row = r0 + (threadIdx.x & 31) / L;
    const bool on = row < n_rows;
    double v = 0.0;
    if (on) {
      const int64_t node = row / D;
      const int64_t a0 = row_ptr[row];
      const int len = (int)(row_ptr[row + 1] - a0);
      const int32_t* cn = col_node + rp_node[node];
      for (int t = sub; t < len; t += L) {
        const int k = t / D;
        const int32_t jj = __ldg(cn + k);
        const int64_t gj = glob ? (int64_t)glob[jj] : (int64_t)jj;
        v = fma(__ldg(A + a0 + t), __ldg(x + D * gj + (t - k * D)), v);
      }
    }
#pragma unroll
    for (int o = 1; o < L; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (on && sub == 0) {
      const int64_t node = row / D;
      const int64_t gi = glob ? (int64_t)glob[node] : node;
      double* dst = y + D * gi + (row - node * D);
      if (shared && shared[node])
        red_add(dst, v);
      else
        *dst = v;
    }
  }
}

}  // namespace fea

using namespace fea;

extern "C" int fea_spmv(fea_mesh* m, int ndof, const int64_t* row_ptr_d, const double* A_d, const double* x_d,
                        double* y_d, const int32_t* glob_d, const uint8_t* shared_d, void* stream) {
  if (!m || !row_ptr_d || !A_d || !x_d || !y_d) return fail(FEA_ERR_ARG, "fea_spmv: null argument");
  if (ndof != 1 && ndof != 3) return fail(FEA_ERR_ARG, "fea_spmv: ndof must be 1 or 3");
  if (!m->rp_node || m->pattern_ndof != ndof)
    return fail(FEA_ERR_ARG, "fea_spmv: build the pattern for this ndof first");
  if (m->n_nodes == 0) return FEA_OK;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  FEA_CUDA(cudaGetDevice(&dev));
  FEA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));

  auto kr = ndof == 1 ? k_spmv_rows<1> : k_spmv_rows<3>;
  int per_sm = 0;
  FEA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kr, 256, 0));
  const int64_t want = ((int64_t)ndof * m->n_nodes * kSpmvLanes + 255) / 256;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * std::max(per_sm, 1)));
  kr<<<grid, 256, 0, s>>>(m->rp_node, m->col_node, row_ptr_d, A_d, x_d, y_d, m->n_nodes, glob_d, shared_d);
  FEA_CUDA(cudaGetLastError());
  return FEA_OK;
}
