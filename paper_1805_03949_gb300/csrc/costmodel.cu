// costmodel.cu -- a small MLP that predicts the cost of work items from
// features of their elements, trained on the per-item timings the persistent
// assembly records, and the longest-processing-time packing of items into
// per-CTA queues.  It is the GPU stand-in for the paper's dynamic load
// balancing (Sec. 4): the cost of an element (a pyramid against a hex, a
// plastic Gauss point against an elastic one) is not known beforehand, so it
// is learned from measurements and used to balance the persistent CTAs.
//
// Network: x (n_in <= 8 features, standardised with the training set's mean
// and population standard deviation) -> 32 tanh -> 32 tanh -> 1, predicting
// the standardised target (log nanoseconds per element).  Loss: mean squared
// error over the training set; optimiser: Adam (beta1 0.9, beta2 0.999,
// eps 1e-8), full batch.  Parameters, FP32, in the order
//   W1 [32][n_in], b1 [32], W2 [32][32], b2 [32], w3 [32], b3.
//
// The network is small (1,313 parameters at n_in = 6): training runs as one
// CTA of 1,024 threads that keeps the parameters in shared memory, pushes the
// training set through in chunks of 256 samples and owns every gradient entry
// in one thread (no atomics); inference is one thread per sample.  There is
// no tensor-core path: at 32 hidden units the products are far too small to
// fill an MMA tile, and the training set (thousands of items) is read once
// per epoch.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <queue>
#include <vector>

#include "element.cuh"
#include "fea_internal.cuh"

struct fea_costmodel {
  int n_in = 0;
  int n_params = 0;
  int64_t step = 0;            // Adam steps taken
  float* params = nullptr;     // device [n_params]
  float* adam_m = nullptr;     // device [n_params]
  float* adam_v = nullptr;     // device [n_params]
  float* scaler = nullptr;     // device [2 * n_in + 2]: x mean, x std, y mean, y std
};

namespace fea {

constexpr int kHid = 32;
constexpr int kMaxIn = 8;
constexpr int kTrainThreads = 1024;
constexpr int kChunk = 256;

__host__ __device__ constexpr int mlp_params(int n_in) { return kHid * n_in + kHid + kHid * kHid + kHid + kHid + 1; }

struct MlpOffsets {
  int W1, b1, W2, b2, w3, b3;
};
__host__ __device__ inline MlpOffsets mlp_offsets(int n_in) {
  MlpOffsets o;
  o.W1 = 0;
  o.b1 = kHid * n_in;
  o.W2 = o.b1 + kHid;
  o.b2 = o.W2 + kHid * kHid;
  o.w3 = o.b2 + kHid;
  o.b3 = o.w3 + kHid;
  return o;
}

// ---------------------------------------------------------------------------
// scaler: mean and population standard deviation of each feature and of the
// target (FP64 sums); a zero deviation is replaced by 1
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_fit_scaler(const float* X, const float* y, int64_t n, int n_in,
                                                     float* scaler) {
  __shared__ double s1[kMaxIn + 1][32], s2[kMaxIn + 1][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int f = 0; f <= n_in; ++f) {
    double a = 0.0, b = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      const double v = f < n_in ? (double)X[i * n_in + f] : (double)y[i];
      a += v;
      b += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
      s1[f][warp] = a;
      s2[f][warp] = b;
    }
  }
  __syncthreads();
  if (threadIdx.x <= n_in) {
    const int f = threadIdx.x;
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += s1[f][w];
      b += s2[f][w];
    }
    const double mean = n > 0 ? a / (double)n : 0.0;
    double var = n > 0 ? b / (double)n - mean * mean : 0.0;
    if (var < 0.0) var = 0.0;
    double sd = sqrt(var);
    if (!(sd > 1e-12 * (fabs(mean) + 1e-30))) sd = 1.0;
    if (f < n_in) {
      scaler[f] = (float)mean;
      scaler[n_in + f] = (float)sd;
    } else {
      scaler[2 * n_in] = (float)mean;
      scaler[2 * n_in + 1] = (float)sd;
    }
  }
}

// ---------------------------------------------------------------------------
// training: one CTA; full-batch gradient of the mean squared error, then an
// Adam step, `epochs` times (epochs = 0: gradient and loss only)
// ---------------------------------------------------------------------------
struct TrainSmem {
  float P[mlp_params(kMaxIn)];
  float X[kChunk][kMaxIn];
  float H1[kChunk][kHid + 1];
  float H2[kChunk][kHid + 1];
  float D2[kChunk][kHid + 1];
  float D1[kChunk][kHid + 1];
  float T[kChunk];      // standardised targets, then dL/dy
  float red[32];
};

__global__ void __launch_bounds__(kTrainThreads) k_mlp_train(float* params, float* adam_m, float* adam_v,
                                                             const float* scaler, const float* X, const float* y,
                                                             int64_t n, int n_in, int epochs, int64_t step0,
                                                             float lr, float* grad_out, float* loss_out) {
  extern __shared__ __align__(16) unsigned char train_raw[];
  TrainSmem& sm = *reinterpret_cast<TrainSmem*>(train_raw);
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const MlpOffsets o = mlp_offsets(n_in);
  const int np = mlp_params(n_in);
  for (int p = t; p < np; p += kTrainThreads) sm.P[p] = params[p];
  // owned parameters: W2[t]; W1[t] (t < 32 n_in); b1, b2, w3 [t] (t < 32); b3 (t == 0)
  const bool ownW1 = t < kHid * n_in, ownV = t < kHid, ownB3 = t == 0;
  float mW2 = adam_m[o.W2 + t], vW2 = adam_v[o.W2 + t];
  float mW1 = ownW1 ? adam_m[o.W1 + t] : 0.f, vW1 = ownW1 ? adam_v[o.W1 + t] : 0.f;
  float mb1 = 0.f, vb1 = 0.f, mb2 = 0.f, vb2 = 0.f, mw3 = 0.f, vw3 = 0.f, mb3 = 0.f, vb3 = 0.f;
  if (ownV) {
    mb1 = adam_m[o.b1 + t]; vb1 = adam_v[o.b1 + t];
    mb2 = adam_m[o.b2 + t]; vb2 = adam_v[o.b2 + t];
    mw3 = adam_m[o.w3 + t]; vw3 = adam_v[o.w3 + t];
  }
  if (ownB3) {
    mb3 = adam_m[o.b3]; vb3 = adam_v[o.b3];
  }
  float xm[kMaxIn], xs[kMaxIn];
  for (int i = 0; i < n_in; ++i) {
    xm[i] = scaler[i];
    xs[i] = 1.0f / scaler[n_in + i];
  }
  const float ym = scaler[2 * n_in], ys = 1.0f / scaler[2 * n_in + 1];
  const float inv_n = n > 0 ? 1.0f / (float)n : 0.0f;
  const int nep = epochs > 0 ? epochs : 1;
  __syncthreads();
  for (int ep = 0; ep < nep; ++ep) {
    float gW2 = 0.f, gW1 = 0.f, gb1 = 0.f, gb2 = 0.f, gw3 = 0.f, gb3 = 0.f, loss = 0.f;
    for (int64_t c0 = 0; c0 < n; c0 += kChunk) {
      const int nb = (int)(n - c0 < kChunk ? n - c0 : kChunk);
      // standardised inputs and targets of the chunk (zero rows past the end)
      for (int k = t; k < kChunk * n_in; k += kTrainThreads) {
        const int s = k / n_in, i = k % n_in;
        sm.X[s][i] = s < nb ? (X[(c0 + s) * n_in + i] - xm[i]) * xs[i] : 0.f;
      }
      if (t < kChunk) sm.T[t] = t < nb ? (y[c0 + t] - ym) * ys : 0.f;
      __syncthreads();
      for (int k = t; k < kChunk * kHid; k += kTrainThreads) {
        const int s = k >> 5, j = k & 31;
        float a = sm.P[o.b1 + j];
        for (int i = 0; i < n_in; ++i) a = fmaf(sm.P[o.W1 + j * n_in + i], sm.X[s][i], a);
        sm.H1[s][j] = tanhf(a);
      }
      __syncthreads();
      for (int k = t; k < kChunk * kHid; k += kTrainThreads) {
        const int s = k >> 5, j = k & 31;
        float a = sm.P[o.b2 + j];
#pragma unroll 8
        for (int i = 0; i < kHid; ++i) a = fmaf(sm.P[o.W2 + j * kHid + i], sm.H1[s][i], a);
        sm.H2[s][j] = tanhf(a);
      }
      __syncthreads();
      // output, residual and dL/dy = 2 (y - t) / n: one warp per sample
      for (int s = warp; s < kChunk; s += kTrainThreads / 32) {
        float v = sm.P[o.w3 + lane] * sm.H2[s][lane];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) {
          const float r = s < nb ? v + sm.P[o.b3] - sm.T[s] : 0.f;
          loss += r * r;
          sm.T[s] = 2.0f * r * inv_n;
        }
      }
      __syncthreads();
      for (int k = t; k < kChunk * kHid; k += kTrainThreads) {
        const int s = k >> 5, j = k & 31;
        const float h = sm.H2[s][j];
        sm.D2[s][j] = sm.T[s] * sm.P[o.w3 + j] * (1.0f - h * h);
      }
      __syncthreads();
      for (int k = t; k < kChunk * kHid; k += kTrainThreads) {
        const int s = k >> 5, i = k & 31;
        float a = 0.f;
#pragma unroll 8
        for (int j = 0; j < kHid; ++j) a = fmaf(sm.D2[s][j], sm.P[o.W2 + j * kHid + i], a);
        const float h = sm.H1[s][i];
        sm.D1[s][i] = a * (1.0f - h * h);
      }
      __syncthreads();
      {  // owned gradient entries
        const int j = t >> 5, i = t & 31;
        for (int s = 0; s < nb; ++s) gW2 = fmaf(sm.D2[s][j], sm.H1[s][i], gW2);
        if (ownW1) {
          const int jj = t / n_in, ii = t % n_in;
          for (int s = 0; s < nb; ++s) gW1 = fmaf(sm.D1[s][jj], sm.X[s][ii], gW1);
        }
        if (ownV)
          for (int s = 0; s < nb; ++s) {
            gb1 += sm.D1[s][t];
            gb2 += sm.D2[s][t];
            gw3 = fmaf(sm.T[s], sm.H2[s][t], gw3);
          }
        if (ownB3)
          for (int s = 0; s < nb; ++s) gb3 += sm.T[s];
      }
      __syncthreads();
    }
    // loss: sum of the per-warp lane-0 partials
    if (lane == 0) sm.red[warp] = loss;
    __syncthreads();
    if (t == 0 && loss_out) {
      float a = 0.f;
      for (int w = 0; w < kTrainThreads / 32; ++w) a += sm.red[w];
      loss_out[0] = a * inv_n;
    }
    if (epochs == 0) {
      grad_out[o.W2 + t] = gW2;
      if (ownW1) grad_out[o.W1 + t] = gW1;
      if (ownV) {
        grad_out[o.b1 + t] = gb1;
        grad_out[o.b2 + t] = gb2;
        grad_out[o.w3 + t] = gw3;
      }
      if (ownB3) grad_out[o.b3] = gb3;
      return;
    }
    // Adam step (bias-corrected) on the owned parameters
    const double st = (double)(step0 + ep + 1);
    const float c1 = (float)(1.0 / (1.0 - pow(0.9, st))), c2 = (float)(1.0 / (1.0 - pow(0.999, st)));
    auto adam = [&](float& p, float& m, float& v, float g) {
      m = 0.9f * m + 0.1f * g;
      v = 0.999f * v + 0.001f * g * g;
      p -= lr * (m * c1) / (sqrtf(v * c2) + 1e-8f);
    };
    __syncthreads();  // every forward read of sm.P of this epoch is done
    adam(sm.P[o.W2 + t], mW2, vW2, gW2);
    if (ownW1) adam(sm.P[o.W1 + t], mW1, vW1, gW1);
    if (ownV) {
      adam(sm.P[o.b1 + t], mb1, vb1, gb1);
      adam(sm.P[o.b2 + t], mb2, vb2, gb2);
      adam(sm.P[o.w3 + t], mw3, vw3, gw3);
    }
    if (ownB3) adam(sm.P[o.b3], mb3, vb3, gb3);
    __syncthreads();
  }
  for (int p = t; p < np; p += kTrainThreads) params[p] = sm.P[p];
  adam_m[o.W2 + t] = mW2;
  adam_v[o.W2 + t] = vW2;
  if (ownW1) {
    adam_m[o.W1 + t] = mW1;
    adam_v[o.W1 + t] = vW1;
  }
  if (ownV) {
    adam_m[o.b1 + t] = mb1; adam_v[o.b1 + t] = vb1;
    adam_m[o.b2 + t] = mb2; adam_v[o.b2 + t] = vb2;
    adam_m[o.w3 + t] = mw3; adam_v[o.w3 + t] = vw3;
  }
  if (ownB3) {
    adam_m[o.b3] = mb3;
    adam_v[o.b3] = vb3;
  }
}

// ---------------------------------------------------------------------------
// inference: one thread per sample; prediction in target units
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_mlp_predict(const float* params, const float* scaler, const float* X,
                                                     int64_t n, int n_in, float* y) {
  __shared__ float P[mlp_params(kMaxIn)];
  const MlpOffsets o = mlp_offsets(n_in);
  const int np = mlp_params(n_in);
  for (int p = threadIdx.x; p < np; p += blockDim.x) P[p] = params[p];
  __syncthreads();
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  float x[kMaxIn];
  for (int i = 0; i < n_in; ++i) x[i] = (X[s * n_in + i] - scaler[i]) / scaler[n_in + i];
  float h1[kHid];
#pragma unroll
  for (int j = 0; j < kHid; ++j) {
    float a = P[o.b1 + j];
    for (int i = 0; i < n_in; ++i) a = fmaf(P[o.W1 + j * n_in + i], x[i], a);
    h1[j] = tanhf(a);
  }
  float out = P[o.b3];
#pragma unroll 4
  for (int j = 0; j < kHid; ++j) {
    float a = P[o.b2 + j];
#pragma unroll
    for (int i = 0; i < kHid; ++i) a = fmaf(P[o.W2 + j * kHid + i], h1[i], a);
    out = fmaf(P[o.w3 + j], tanhf(a), out);
  }
  y[s] = out * scaler[2 * n_in + 1] + scaler[2 * n_in];
}

// ---------------------------------------------------------------------------
// item features: per element, the one-hot type (4), the fraction of its
// points that yielded in the committed state (alpha_n > 0), and the Frobenius
// norm of the small strain sym(grad u) at the element's reference centroid;
// per item, the mean over its elements.  One CTA per item.
// ---------------------------------------------------------------------------
struct FeatArgs {
  const WorkItem* items;
  int64_t n_items;
  const double* coords;
  const double* u;          // may be nullptr (strain norm 0)
  const double* state_in;   // may be nullptr (yield fraction 0)
  const int32_t* tconn[kNumTypes];
  const int32_t* ids[kNumTypes];
  float* X;                 // [n_items][6]
};

__device__ __forceinline__ void centroid_dN(int type, int a, double d[3]) {
  // reference centroids: tet (1/4,1/4,1/4), pyramid (0,0,1/4) on the rational
  // basis, prism (1/3,1/3,0), hex (0,0,0)
  switch (type) {
    case FEA_TET4:
      d[0] = a == 1 ? 1.0 : a == 0 ? -1.0 : 0.0;
      d[1] = a == 2 ? 1.0 : a == 0 ? -1.0 : 0.0;
      d[2] = a == 3 ? 1.0 : a == 0 ? -1.0 : 0.0;
      return;
    case FEA_PYR5: {
      if (a == 4) {
        d[0] = d[1] = 0.0;
        d[2] = 1.0;
        return;
      }
      const double sx = (a == 1 || a == 2) ? 1.0 : -1.0, sy = (a >= 2) ? 1.0 : -1.0;
      const double z = 0.25, tt = 1.0 - z;  // x = y = 0: u = v = 1 - z
      d[0] = sx * tt / (4.0 * tt);
      d[1] = sy * tt / (4.0 * tt);
      d[2] = (tt * tt - tt * (2.0 * tt)) / (4.0 * tt * tt);
      return;
    }
    case FEA_PRISM6: {
      const int k = a % 3;
      const double L = 1.0 / 3.0, h = 0.5, hz = a < 3 ? -0.5 : 0.5;
      d[0] = (k == 0 ? -1.0 : k == 1 ? 1.0 : 0.0) * h;
      d[1] = (k == 0 ? -1.0 : k == 2 ? 1.0 : 0.0) * h;
      d[2] = L * hz;
      return;
    }
    default: {
      const int bx = ((a + 1) >> 1) & 1, by = (a >> 1) & 1, bz = a >> 2;
      d[0] = 0.125 * (bx ? 1.0 : -1.0);
      d[1] = 0.125 * (by ? 1.0 : -1.0);
      d[2] = 0.125 * (bz ? 1.0 : -1.0);
      return;
    }
  }
}

__global__ void __launch_bounds__(128) k_item_features(const __grid_constant__ FeatArgs F) {
  const int64_t item = blockIdx.x;
  if (item >= F.n_items) return;
  const WorkItem it = F.items[item];
  const int type = it.entry;
  const int nn = nodes_of(type);
  const int nq = type == FEA_TET4 ? 4 : type == FEA_PRISM6 ? 6 : 8;
  float yl = 0.f, sn = 0.f;
  for (int k = threadIdx.x; k < it.count; k += blockDim.x) {
    const int64_t g = (int64_t)it.first + k;
    const int32_t* en = F.tconn[type] + g * nn;
    const int64_t id = F.ids[type] ? (int64_t)F.ids[type][g] : g;
    if (F.state_in) {
      int c = 0;
      for (int q = 0; q < nq; ++q) c += F.state_in[(id * 8 + q) * 7 + 6] > 0.0;
      yl += (float)c / (float)nq;
    }
    if (F.u) {
      double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, Gu[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
      double dN[8][3];
      const double* x0 = F.coords + 3 * (int64_t)en[0];
      for (int a = 0; a < nn; ++a) {
        centroid_dN(type, a, dN[a]);
        const double* xa = F.coords + 3 * (int64_t)en[a];
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) J[i][j] += (xa[i] - x0[i]) * dN[a][j];
      }
      double C[3][3];
      cofactors(J, C);
      const double det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
      if (det > 0.0) {
        for (int a = 0; a < nn; ++a) {
          const double* ua = F.u + 3 * (int64_t)en[a];
          double g[3];
          for (int i = 0; i < 3; ++i) g[i] = (dN[a][0] * C[i][0] + dN[a][1] * C[i][1] + dN[a][2] * C[i][2]) / det;
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) Gu[i][j] += ua[i] * g[j];
        }
        double s2 = 0.0;
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) {
            const double e = 0.5 * (Gu[i][j] + Gu[j][i]);
            s2 += e * e;
          }
        sn += (float)sqrt(s2);
      }
    }
  }
  __shared__ float r1[4], r2[4];
  for (int o = 16; o > 0; o >>= 1) {
    yl += __shfl_xor_sync(0xffffffffu, yl, o);
    sn += __shfl_xor_sync(0xffffffffu, sn, o);
  }
  if ((threadIdx.x & 31) == 0) {
    r1[threadIdx.x >> 5] = yl;
    r2[threadIdx.x >> 5] = sn;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const float inv = it.count > 0 ? 1.0f / (float)it.count : 0.f;
    float* x = F.X + item * 6;
    for (int tt = 0; tt < 4; ++tt) x[tt] = tt == type ? 1.f : 0.f;
    x[4] = (r1[0] + r1[1] + r1[2] + r1[3]) * inv;
    x[5] = (r2[0] + r2[1] + r2[2] + r2[3]) * inv;
  }
}

}  // namespace fea

using namespace fea;

extern "C" {

int fea_costmodel_create(int n_in, const float* params_h, fea_costmodel** out) {
  if (!params_h || !out) return fail(FEA_ERR_ARG, "fea_costmodel_create: null argument");
  if (n_in < 1 || n_in > kMaxIn) return fail(FEA_ERR_ARG, "fea_costmodel_create: n_in must be in [1, 8]");
  fea_costmodel* m = new fea_costmodel();
  m->n_in = n_in;
  m->n_params = mlp_params(n_in);
  const size_t pb = (size_t)m->n_params * sizeof(float);
  if (cudaMalloc(&m->params, pb) != cudaSuccess || cudaMalloc(&m->adam_m, pb) != cudaSuccess ||
      cudaMalloc(&m->adam_v, pb) != cudaSuccess ||
      cudaMalloc(&m->scaler, (2 * n_in + 2) * sizeof(float)) != cudaSuccess) {
    cudaFree(m->params); cudaFree(m->adam_m); cudaFree(m->adam_v); cudaFree(m->scaler);
    delete m;
    return fail(FEA_ERR_OOM, "fea_costmodel_create: cudaMalloc failed");
  }
  std::vector<float> sc(2 * n_in + 2, 0.0f);
  for (int i = 0; i < n_in; ++i) sc[n_in + i] = 1.0f;
  sc[2 * n_in + 1] = 1.0f;
  if (cudaMemcpy(m->params, params_h, pb, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(m->adam_m, 0, pb) != cudaSuccess || cudaMemset(m->adam_v, 0, pb) != cudaSuccess ||
      cudaMemcpy(m->scaler, sc.data(), sc.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(m->params); cudaFree(m->adam_m); cudaFree(m->adam_v); cudaFree(m->scaler);
    delete m;
    return fail(FEA_ERR_CUDA, "fea_costmodel_create: initial copy failed");
  }
  *out = m;
  return FEA_OK;
}

int fea_costmodel_destroy(fea_costmodel* m) {
  if (!m) return fail(FEA_ERR_ARG, "fea_costmodel_destroy: null handle");
  cudaDeviceSynchronize();
  cudaFree(m->params); cudaFree(m->adam_m); cudaFree(m->adam_v); cudaFree(m->scaler);
  delete m;
  return FEA_OK;
}

int fea_costmodel_get_params(const fea_costmodel* m, float* params_h, float* scaler_h) {
  if (!m) return fail(FEA_ERR_ARG, "fea_costmodel_get_params: null handle");
  if (params_h) FEA_CUDA(cudaMemcpy(params_h, m->params, m->n_params * sizeof(float), cudaMemcpyDeviceToHost));
  if (scaler_h) FEA_CUDA(cudaMemcpy(scaler_h, m->scaler, (2 * m->n_in + 2) * sizeof(float), cudaMemcpyDeviceToHost));
  return FEA_OK;
}

int fea_costmodel_fit_scaler(fea_costmodel* m, const float* X_d, const float* y_d, int64_t n, void* stream) {
  if (!m || (n > 0 && (!X_d || !y_d)) || n < 0) return fail(FEA_ERR_ARG, "fea_costmodel_fit_scaler: bad argument");
  k_fit_scaler<<<1, 1024, 0, (cudaStream_t)stream>>>(X_d, y_d, n, m->n_in, m->scaler);
  FEA_CUDA(cudaGetLastError());
  return FEA_OK;
}

static int train_launch(fea_costmodel* m, const float* X_d, const float* y_d, int64_t n, int epochs, float lr,
                        float* grad_d, float* loss_d, cudaStream_t s) {
  const size_t smem = sizeof(TrainSmem);
  FEA_CUDA(cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_mlp_train<<<1, kTrainThreads, smem, s>>>(m->params, m->adam_m, m->adam_v, m->scaler, X_d, y_d, n, m->n_in,
                                             epochs, m->step, lr, grad_d, loss_d);
  FEA_CUDA(cudaGetLastError());
  return FEA_OK;
}

int fea_costmodel_grad(fea_costmodel* m, const float* X_d, const float* y_d, int64_t n, float* grad_d, float* loss_d,
                       void* stream) {
  if (!m || !X_d || !y_d || !grad_d || n <= 0) return fail(FEA_ERR_ARG, "fea_costmodel_grad: bad argument");
  return train_launch(m, X_d, y_d, n, 0, 0.0f, grad_d, loss_d, (cudaStream_t)stream);
}

int fea_costmodel_train(fea_costmodel* m, const float* X_d, const float* y_d, int64_t n, int epochs, float lr,
                        float* loss_d, void* stream) {
  if (!m || !X_d || !y_d || n <= 0 || epochs < 1) return fail(FEA_ERR_ARG, "fea_costmodel_train: bad argument");
  if (!(lr > 0.0f)) return fail(FEA_ERR_ARG, "fea_costmodel_train: lr must be positive");
  const int rc = train_launch(m, X_d, y_d, n, epochs, lr, nullptr, loss_d, (cudaStream_t)stream);
  if (rc == FEA_OK) m->step += epochs;
  return rc;
}

int fea_costmodel_predict(const fea_costmodel* m, const float* X_d, int64_t n, float* y_d, void* stream) {
  if (!m || (n > 0 && (!X_d || !y_d)) || n < 0) return fail(FEA_ERR_ARG, "fea_costmodel_predict: bad argument");
  if (n == 0) return FEA_OK;
  k_mlp_predict<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(m->params, m->scaler, X_d, n, m->n_in, y_d);
  FEA_CUDA(cudaGetLastError());
  return FEA_OK;
}

int fea_item_features(fea_mesh* mesh, int chunk, const double* u_d, const double* state_in_d, float* X_d,
                      void* stream) {
  if (!mesh || !X_d) return fail(FEA_ERR_ARG, "fea_item_features: null argument");
  if (chunk < 0 || chunk > (1 << 24)) return fail(FEA_ERR_ARG, "fea_item_features: chunk must be in [0, 2^24]");
  std::vector<WorkItem> h;
  const int ch = chunk > 0 ? chunk : 128;
  for (int t = 0; t < kNumTypes; ++t)
    for (int64_t f = 0; f < mesh->group[t].n; f += ch) {
      WorkItem w;
      w.entry = t;
      w.first = (int32_t)f;
      w.count = (int32_t)std::min<int64_t>(ch, mesh->group[t].n - f);
      w.pad = 0;
      h.push_back(w);
    }
  if (h.empty()) return FEA_OK;
  WorkItem* d = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  FEA_CUDA(cudaMallocAsync((void**)&d, h.size() * sizeof(WorkItem), s));
  FEA_CUDA(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, s));
  FeatArgs F;
  std::memset(&F, 0, sizeof(F));
  F.items = d;
  F.n_items = (int64_t)h.size();
  F.coords = mesh->coords;
  F.u = u_d;
  F.state_in = state_in_d;
  for (int t = 0; t < kNumTypes; ++t) {
    F.tconn[t] = mesh->group[t].conn;
    F.ids[t] = mesh->group[t].ids;
  }
  F.X = X_d;
  k_item_features<<<(unsigned)h.size(), 128, 0, s>>>(F);
  cudaError_t e = cudaGetLastError();
  cudaFreeAsync(d, s);
  FEA_CUDA(cudaStreamSynchronize(s));  // the host list h must outlive the copy
  if (e != cudaSuccess) return cuda_fail(e, "k_item_features");
  return FEA_OK;
}

int fea_pack_lpt(const double* cost_h, int64_t n_items, int n_queues, int32_t* queue_h, int64_t* queue_off_h,
                 double* load_h) {
  if ((n_items > 0 && !cost_h) || !queue_h || !queue_off_h || n_queues < 1 || n_items < 0)
    return fail(FEA_ERR_ARG, "fea_pack_lpt: bad argument");
  // longest processing time first: items by decreasing cost (ties: lower id
  // first), each onto the queue with the least load so far (ties: lower queue)
  std::vector<int32_t> order(n_items);
  for (int64_t i = 0; i < n_items; ++i) order[i] = (int32_t)i;
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return cost_h[a] > cost_h[b]; });
  using Slot = std::pair<double, int>;
  std::priority_queue<Slot, std::vector<Slot>, std::greater<Slot>> heap;
  for (int q = 0; q < n_queues; ++q) heap.push({0.0, q});
  std::vector<int> owner(n_items);
  std::vector<double> load(n_queues, 0.0);
  for (int64_t k = 0; k < n_items; ++k) {
    Slot sl = heap.top();
    heap.pop();
    owner[order[k]] = sl.second;
    sl.first += cost_h[order[k]];
    load[sl.second] = sl.first;
    heap.push(sl);
  }
  // queues in assignment order (longest first within a queue)
  std::vector<int64_t> cnt(n_queues + 1, 0);
  for (int64_t i = 0; i < n_items; ++i) ++cnt[owner[i] + 1];
  for (int q = 0; q < n_queues; ++q) cnt[q + 1] += cnt[q];
  for (int q = 0; q <= n_queues; ++q) queue_off_h[q] = cnt[q];
  std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
  for (int64_t k = 0; k < n_items; ++k) queue_h[pos[owner[order[k]]]++] = order[k];
  if (load_h)
    for (int q = 0; q < n_queues; ++q) load_h[q] = load[q];
  return FEA_OK;
}

}  // extern "C"
