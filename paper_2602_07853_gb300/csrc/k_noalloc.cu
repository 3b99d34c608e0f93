// Allocation-free particle sort (mpml_sort_particles_noalloc, declared in
// include/mpml.h).
//
// Who needs it: callers that must not call cudaMalloc at the point where they
// sort particles -- an application that hands all device memory to its own
// arena up front and forbids other allocations, or a time-critical loop that
// cannot afford cudaMalloc's implicit device-wide synchronisation while other
// streams are busy.  A library context cannot serve them: mpml_create and
// mpml_resample allocate and grow their buffers.
//
// What it computes: the order in which mpml_resample sorts particles -- by
// the brick-major key of the base centre floor(x/dx - 1/2), ties by input
// index -- and optionally each sorted particle's key.  It is a variant of the
// resample's binning and counting sort that keys on the dense brick grid
// instead of the compacted active bricks (both orders are the same because
// the compaction keeps brick order), so that its scratch has a size fixed by
// the grid alone.
//
// Scratch: one file-scope device array of MPML_NOALLOC_MAX_SLOTS counters,
// as many start offsets, the scan's block sums and a status word (about
// 16 MiB).  The CUDA runtime places it in a device's memory when it loads the
// library's code there -- by default lazily, at the first use of the library
// on that device, which may be this entry point's first call -- and it stays
// until the process exits.  So the first call on a device (or any earlier
// library call there) must come before an arena claims the device's memory
// and before any stream capture.  The host never dereferences the symbol:
// every call asks cudaGetSymbolAddress (a host-side lookup that allocates
// nothing once the code is loaded) for its address on the current device and
// passes that to the kernels, so the address stays right after a
// cudaDeviceReset reloads the code.  Every call clears the counters and the
// status word it uses, so a call never sees a previous call's data; but all
// calls on one device share the array, so two calls whose kernels overlap on
// the GPU (different streams, or different host threads) race and give wrong
// results.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <cstdint>

#include "mpml.h"

namespace {

constexpr int64_t NA_MAX_SLOTS = MPML_NOALLOC_MAX_SLOTS;
constexpr int NA_SCAN_T = 1024;                  // threads per scan block
constexpr int NA_SCAN_E = 2 * NA_SCAN_T;         // slots per scan block
constexpr int64_t NA_NBLK_MAX = NA_MAX_SLOTS / NA_SCAN_E;
static_assert(NA_MAX_SLOTS % NA_SCAN_E == 0, "slot capacity must be a multiple of the scan block");
static_assert(NA_NBLK_MAX <= NA_SCAN_T, "block sums must fit one scan block");

// int offsets into the scratch array (each part starts on a 256-byte boundary)
constexpr int64_t NA_OFF_CNT = 0;                           // [NA_MAX_SLOTS] counts, then cursors
constexpr int64_t NA_OFF_START = NA_MAX_SLOTS;              // [NA_MAX_SLOTS + 1] exclusive offsets
constexpr int64_t NA_OFF_BSUM = 2 * NA_MAX_SLOTS + 64;      // [NA_NBLK_MAX + 1] scan block sums
constexpr int64_t NA_OFF_STATUS = NA_OFF_BSUM + NA_NBLK_MAX + 64;
constexpr int64_t NA_INTS = NA_OFF_STATUS + 64;

constexpr int NA_ST_OUT_OF_DOMAIN = 1;
constexpr int NA_ST_NONFINITE = 2;

static __device__ __align__(256) int na_scratch[NA_INTS];

struct NaGrid {
  int n[3];
  int NB[3];
  double inv_dx;
};

// Dense brick-major key of the particle's base centre, or -1 (status set)
// when a coordinate is not finite or the 2x2x2 centre stencil leaves the grid.
// x/dx - 1/2 is rounded step by step (no fused multiply-add), as in the
// library's other binning kernels, so that both agree on every particle.
__device__ __forceinline__ int64_t na_key(const NaGrid& g, const double xa[3], int* status) {
  int b[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (!isfinite(xa[a])) {
      atomicOr(status, NA_ST_NONFINITE);
      return -1;
    }
    const double s = __dsub_rn(__dmul_rn(xa[a], g.inv_dx), 0.5);
    const double fl = floor(s);
    if (fl < 0.0 || fl + 1.0 > (double)(g.n[a] - 1)) {
      atomicOr(status, NA_ST_OUT_OF_DOMAIN);
      return -1;
    }
    b[a] = (int)fl;
  }
  const int64_t brick = ((int64_t)(b[2] >> 3) * g.NB[1] + (b[1] >> 3)) * g.NB[0] + (b[0] >> 3);
  return brick * 512 + (b[2] & 7) * 64 + (b[1] & 7) * 8 + (b[0] & 7);
}

template <typename T>
__device__ __forceinline__ int64_t na_particle_key(const NaGrid& g, const T* x, int64_t p, int* status) {
  const double xa[3] = {(double)x[3 * p], (double)x[3 * p + 1], (double)x[3 * p + 2]};
  return na_key(g, xa, status);
}

__global__ void k_na_clear(int* cnt, int64_t nslots, int* status) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *status = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nslots; i += (int64_t)gridDim.x * blockDim.x)
    cnt[i] = 0;
}

template <typename T>
__global__ void k_na_count(int64_t np, const T* __restrict__ x, NaGrid g, int* cnt, int* status) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const int64_t k = na_particle_key(g, x, p, status);
  if (k >= 0) atomicAdd(&cnt[k], 1);
}

// Exclusive prefix of v over the block; *total receives the block's sum.
__device__ int na_block_scan(int v, int* total) {
  __shared__ int warp_sum[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_sum[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int w = lane < nw ? warp_sum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    warp_sum[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  const int ex = incl - v + (wid > 0 ? warp_sum[wid - 1] : 0);
  *total = warp_sum[nw - 1];
  __syncthreads();
  return ex;
}

__global__ void k_na_scan_blocks(const int* cnt, int64_t nslots, int* bsum) {
  const int64_t i0 = (int64_t)blockIdx.x * NA_SCAN_E + 2 * threadIdx.x;
  const int v = (i0 < nslots ? cnt[i0] : 0) + (i0 + 1 < nslots ? cnt[i0 + 1] : 0);
  int total;
  na_block_scan(v, &total);
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// one block: block sums -> their exclusive offsets; start[nslots] = total
__global__ void k_na_scan_sums(int* bsum, int nblk, int* start, int64_t nslots) {
  const int v = (int)threadIdx.x < nblk ? bsum[threadIdx.x] : 0;
  int total;
  const int ex = na_block_scan(v, &total);
  if ((int)threadIdx.x < nblk) bsum[threadIdx.x] = ex;
  if (threadIdx.x == 0) start[nslots] = total;
}

// start = exclusive scan of the counts; the counts become scatter cursors
__global__ void k_na_scan_apply(int* cnt, int64_t nslots, const int* bsum, int* start) {
  const int64_t i0 = (int64_t)blockIdx.x * NA_SCAN_E + 2 * threadIdx.x;
  const int a = i0 < nslots ? cnt[i0] : 0;
  const int b = i0 + 1 < nslots ? cnt[i0 + 1] : 0;
  int total;
  const int ex = na_block_scan(a + b, &total) + bsum[blockIdx.x];
  if (i0 < nslots) start[i0] = cnt[i0] = ex;
  if (i0 + 1 < nslots) start[i0 + 1] = cnt[i0 + 1] = ex + a;
}

template <typename T>
__global__ void k_na_scatter(int64_t np, const T* __restrict__ x, NaGrid g, int* cursor, int32_t* perm,
                             int* status) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const int64_t k = na_particle_key(g, x, p, status);
  if (k >= 0) perm[atomicAdd(&cursor[k], 1)] = (int32_t)p;
}

// Within one centre the scatter order is arbitrary: restore input order.
// A thread sorts the segment of its centre in place when it is short (at most
// NA_SEG_SHORT particles, insertion sort); longer segments are queued in shared
// memory and sorted by the whole block: up to NA_SEG_SMEM particles are staged
// in shared memory and each goes to its rank (the indices in a segment are
// distinct), O(k^2 / 256) per block; a segment longer than that (compressed
// material with thousands of particles in one centre) falls back to one
// thread's insertion sort, O(k^2).
constexpr int NA_SEG_SHORT = 32;
constexpr int NA_SEG_SMEM = 4096;

__global__ void __launch_bounds__(256) k_na_order_segments(int64_t nslots, const int* start, int32_t* perm,
                                                           int64_t* keys) {
  __shared__ int64_t s_queue[256];
  __shared__ int s_nq;
  __shared__ int32_t s_seg[NA_SEG_SMEM];
  if (threadIdx.x == 0) s_nq = 0;
  __syncthreads();
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nslots) {
    const int s = start[k], e = start[k + 1];
    if (e - s <= NA_SEG_SHORT) {
      for (int i = s + 1; i < e; ++i) {
        const int32_t v = perm[i];
        int j = i - 1;
        while (j >= s && perm[j] > v) {
          perm[j + 1] = perm[j];
          --j;
        }
        perm[j + 1] = v;
      }
      if (keys)
        for (int i = s; i < e; ++i) keys[i] = k;
    } else {
      s_queue[atomicAdd(&s_nq, 1)] = k;
    }
  }
  __syncthreads();
  const int nq = s_nq;
  for (int qi = 0; qi < nq; ++qi) {
    const int64_t kk = s_queue[qi];
    const int s = start[kk], e = start[kk + 1], len = e - s;
    if (len <= NA_SEG_SMEM) {
      for (int i = threadIdx.x; i < len; i += blockDim.x) s_seg[i] = perm[s + i];
      __syncthreads();
      for (int i = threadIdx.x; i < len; i += blockDim.x) {
        const int32_t v = s_seg[i];
        int r = 0;
        for (int j = 0; j < len; ++j) r += s_seg[j] < v ? 1 : 0;
        perm[s + r] = v;
      }
      __syncthreads();  // s_seg is reused by the next queued segment
    } else if (threadIdx.x == 0) {
      for (int i = s + 1; i < e; ++i) {
        const int32_t v = perm[i];
        int j = i - 1;
        while (j >= s && perm[j] > v) {
          perm[j + 1] = perm[j];
          --j;
        }
        perm[j + 1] = v;
      }
    }
    if (keys)
      for (int i = s + (int)threadIdx.x; i < e; i += blockDim.x) keys[i] = kk;
  }
}

// Device address of the scratch array on the current device (looked up on
// every call: cheap, allocation-free once the code is loaded, and never stale).
int na_scratch_base(int** out) {
  int* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress((void**)&p, na_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    return MPML_ERR_CUDA;
  }
  *out = p;
  return MPML_OK;
}

unsigned na_blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename T>
int na_sort(const NaGrid& g, int64_t nslots, const T* x, int64_t np, int32_t* perm, int64_t* keys,
            cudaStream_t s, int* base) {
  int* cnt = base + NA_OFF_CNT;
  int* start = base + NA_OFF_START;
  int* bsum = base + NA_OFF_BSUM;
  int* status = base + NA_OFF_STATUS;
  const int nblk = (int)na_blocks(nslots, NA_SCAN_E);
  const unsigned clear_blocks = na_blocks(nslots, 256) < 152u * 8u ? na_blocks(nslots, 256) : 152u * 8u;
  k_na_clear<<<clear_blocks, 256, 0, s>>>(cnt, nslots, status);
  k_na_count<T><<<na_blocks(np, 256), 256, 0, s>>>(np, x, g, cnt, status);
  k_na_scan_blocks<<<nblk, NA_SCAN_T, 0, s>>>(cnt, nslots, bsum);
  k_na_scan_sums<<<1, NA_SCAN_T, 0, s>>>(bsum, nblk, start, nslots);
  k_na_scan_apply<<<nblk, NA_SCAN_T, 0, s>>>(cnt, nslots, bsum, start);
  k_na_scatter<T><<<na_blocks(np, 256), 256, 0, s>>>(np, x, g, cnt, perm, status);
  k_na_order_segments<<<na_blocks(nslots, 256), 256, 0, s>>>(nslots, start, perm, keys);
  if (cudaGetLastError() != cudaSuccess) return MPML_ERR_CUDA;
  int hstatus = 0;
  if (cudaMemcpyAsync(&hstatus, status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return MPML_ERR_CUDA;
  }
  if (hstatus & NA_ST_NONFINITE) return MPML_ERR_NONFINITE;
  if (hstatus & NA_ST_OUT_OF_DOMAIN) return MPML_ERR_OUT_OF_DOMAIN;
  return MPML_OK;
}

}  // namespace

extern "C" int mpml_sort_particles_noalloc(const int n[3], double inv_dx, int precision, const void* x,
                                           int64_t n_particles, int32_t* perm, int64_t* keys, void* stream) {
  if (!n || !(inv_dx > 0.0) || !std::isfinite(inv_dx)) return MPML_ERR_ARG;
  if (precision != MPML_FP32 && precision != MPML_FP64) return MPML_ERR_ARG;
  if (n_particles < 0 || n_particles > INT32_MAX) return MPML_ERR_ARG;
  if (n_particles > 0 && (!x || !perm)) return MPML_ERR_ARG;
  NaGrid g;
  int64_t nslots = 512;
  for (int a = 0; a < 3; ++a) {
    if (n[a] < 2) return MPML_ERR_ARG;
    g.n[a] = n[a];
    g.NB[a] = (n[a] >> 3) + 1;
    nslots *= g.NB[a];
    if (nslots > NA_MAX_SLOTS) return MPML_ERR_TOO_LARGE;
  }
  g.inv_dx = inv_dx;
  if (n_particles == 0) return MPML_OK;
  int* base = nullptr;
  const int rc = na_scratch_base(&base);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == MPML_FP64)
    return na_sort<double>(g, nslots, (const double*)x, n_particles, perm, keys, s, base);
  return na_sort<float>(g, nslots, (const float*)x, n_particles, perm, keys, s, base);
}
