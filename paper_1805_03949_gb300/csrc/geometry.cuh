// geometry.cuh -- per-element geometry records (see geometry.cu).
#pragma once

#include <cuda_runtime.h>

#include "fea_gb300.h"

namespace fea {

// record of one element: g^ [8 q][8 a][3], then W [8], then K [8]
constexpr int kRecStride = 208;
constexpr int kRecW = 192;
constexpr int kRecK = 200;

// Evaluate the records of every element for this operator (stream-ordered,
// into a buffer owned by the mesh handle, one per precision).
int geometry_pass(const fea_operator* op, fea_mesh* m, cudaStream_t s, void** records, int* launched);
int geometry_launches(const fea_mesh* m);

}  // namespace fea
