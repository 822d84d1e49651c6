// Degree order of the stored sources and destination order of the hub sources'
// edges (dualip_create, dualip_get_primal).
//
// A problem whose source degrees spread widely is stored with its sources in
// order of increasing degree.  The pass takes sources in batches of eight
// consecutive ones and sizes the lane groups of a batch by its largest span,
// so similar degrees within a batch keep its lanes busy.  The problem is
// separable by source (Section 3.1: the projection is one simplex per
// source), so the order changes no per-source result: A x is summed exactly,
// and only the order of the objective's partial sums moves.
//
// Hub sources (the multi-block class) are, besides, stored with their edges
// in order of destination: a source's simplex is the same in any order of
// its edges, and sorted ids let a warp's mu gathers share sectors.
//
// These kernels move whole source segments between the caller's edge order
// and the stored one: one warp per stored source, its lanes over the
// segment's edges (coalesced on both sides).
#include <cuda_bf16.h>

#include "internal.h"

namespace dualip {
namespace {

int warps_grid(int64_t sources) {
  int64_t g = (32 * sources + 255) / 256;  // 8 warps per 256-thread block
  if (g < 1) g = 1;
  if (g > 8192) g = 8192;
  return (int)g;
}

__device__ __forceinline__ uint32_t bf16_pair(float c, float a) {
  const uint32_t cb = __bfloat16_as_ushort(__float2bfloat16_rn(c));
  const uint32_t ab = __bfloat16_as_ushort(__float2bfloat16_rn(a));
  return cb | (ab << 16);
}

// Stored source i is the caller's source m.src_of[i]: its edges start at
// m.orig_off[m.src_of[i]] in the caller's arrays and at m.off[i] in storage.
__global__ void renumber_seg_kernel(const int32_t* __restrict__ in, int32_t* __restrict__ out,
                                    const int32_t* __restrict__ new_of, SegMap m, int32_t J,
                                    DeviceStatus* st) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < m.I; i += nw) {
    const int64_t o = m.off[i], n = m.off[i + 1] - o, g = m.orig_off[m.src_of[i]];
    for (int64_t k = lane; k < n; k += 32) {
      const int32_t j = in[g + k];
      if (j < 0 || j >= J) {
        atomicOr(&st->err, kErrBounds);
        out[o + k] = 0;
        continue;
      }
      out[o + k] = new_of[j];
    }
  }
}

template <bool BF16>
__global__ void pack_seg_kernel(const float* __restrict__ c, const float* __restrict__ a,
                                void* __restrict__ out, SegMap m) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < m.I; i += nw) {
    const int64_t o = m.off[i], n = m.off[i + 1] - o, g = m.orig_off[m.src_of[i]];
    for (int64_t k = lane; k < n; k += 32) {
      if (BF16)
        static_cast<uint32_t*>(out)[o + k] = bf16_pair(c[g + k], a[g + k]);
      else
        static_cast<float2*>(out)[o + k] = make_float2(c[g + k], a[g + k]);
    }
  }
}

// The inverse copy, for the primal x: from stored order to the caller's.
__global__ void unpermute_seg_kernel(const float* __restrict__ in, float* __restrict__ out,
                                     SegMap m) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < m.I; i += nw) {
    const int64_t o = m.off[i], n = m.off[i + 1] - o, g = m.orig_off[m.src_of[i]];
    for (int64_t k = lane; k < n; k += 32) out[g + k] = in[o + k];
  }
}

// A permutation within one segment (the destination order of a hub source):
// out[k] = in[perm[k]], and its inverse for the primal x.
template <typename T>
__global__ void gather_perm_kernel(const T* __restrict__ in, T* __restrict__ out,
                                   const uint32_t* __restrict__ perm, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += stride)
    out[k] = in[perm[k]];
}

__global__ void scatter_perm_kernel(const float* __restrict__ in, float* __restrict__ out,
                                    const uint32_t* __restrict__ perm, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += stride)
    out[perm[k]] = in[k];
}

int elems_grid(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g < 1) g = 1;
  if (g > 8192) g = 8192;
  return (int)g;
}

}  // namespace

cudaError_t launch_gather_perm(const void* in, void* out, const uint32_t* perm, int64_t n,
                               int elem_bytes, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (elem_bytes == 8)
    gather_perm_kernel<uint2><<<elems_grid(n), 256, 0, s>>>(static_cast<const uint2*>(in),
                                                            static_cast<uint2*>(out), perm, n);
  else if (elem_bytes == 4)
    gather_perm_kernel<uint32_t><<<elems_grid(n), 256, 0, s>>>(
        static_cast<const uint32_t*>(in), static_cast<uint32_t*>(out), perm, n);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_scatter_perm(const float* in, float* out, const uint32_t* perm, int64_t n,
                                cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  scatter_perm_kernel<<<elems_grid(n), 256, 0, s>>>(in, out, perm, n);
  return cudaGetLastError();
}

cudaError_t launch_renumber_seg(const int32_t* dst_in, int32_t* dst_out, const int32_t* new_of,
                                const SegMap& m, int32_t J, DeviceStatus* st, cudaStream_t s) {
  renumber_seg_kernel<<<warps_grid(m.I), 256, 0, s>>>(dst_in, dst_out, new_of, m, J, st);
  return cudaGetLastError();
}

cudaError_t launch_pack_seg(const float* c, const float* a, int storage, void* out,
                            const SegMap& m, cudaStream_t s) {
  if (storage == DUALIP_EDGE_BF16)
    pack_seg_kernel<true><<<warps_grid(m.I), 256, 0, s>>>(c, a, out, m);
  else
    pack_seg_kernel<false><<<warps_grid(m.I), 256, 0, s>>>(c, a, out, m);
  return cudaGetLastError();
}

cudaError_t launch_unpermute_seg(const float* in, float* out, const SegMap& m, cudaStream_t s) {
  unpermute_seg_kernel<<<warps_grid(m.I), 256, 0, s>>>(in, out, m);
  return cudaGetLastError();
}

}  // namespace dualip
