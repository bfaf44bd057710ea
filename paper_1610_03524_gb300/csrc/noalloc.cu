// noalloc.cu -- rank/select directory of a bitvector without any device
// allocation (rs_dir_build_static in include/wavelet.h).
//
// Some callers cannot allocate device memory at the moment they need the
// directory: code that runs while another component owns every byte of the
// device through its own memory manager, latency-critical paths where an
// allocation call may wait for the whole device, or hosts that forbid driver
// allocations after start-up.  For them this file keeps the build's only
// scratch buffer (per-superblock zero counts and the scan's block sums) in a
// file-scope __device__ array, reserved once when the library is loaded on a
// device and kept until the process exits.  The caller provides the input
// bits and the output arrays; nothing here calls cudaMalloc, cudaFree or any
// allocating routine.
//
// The scratch array is shared by every call: two calls whose kernels overlap
// on the GPU (different streams, or different host threads) race on it.
// Calls must be ordered, e.g. issued on one stream.
#include <cstdio>
#include <mutex>

#include "wt_host.h"
#include "wt_internal.cuh"

namespace wtk {

// Largest bitvector accepted: 2^30 bits (2^19 superblocks of 2048 bits).
constexpr uint64_t NOALLOC_MAX_BITS = 1ull << 30;
constexpr uint64_t NOALLOC_MAX_SB = NOALLOC_MAX_BITS / 2048;
// the scan below: 1024 threads x 4 counts per block
constexpr int NA_BT = 1024, NA_PER = 4, NA_CH = NA_BT * NA_PER;
// superblock zero counts, scanned in place (+1 total), then the scan's block
// sums (one per block of NA_CH counts, + total)
constexpr uint64_t NOALLOC_SCRATCH = (NOALLOC_MAX_SB + 1) + (NOALLOC_MAX_SB / NA_CH + 2);

static __device__ __align__(256) uint64_t g_noalloc_scratch[NOALLOC_SCRATCH];

namespace {

// Host-side device address of g_noalloc_scratch on device `dev` (the symbol
// name itself is only a host stand-in).  Looked up with that device current
// on every call outside stream capture, so the address stays right after a
// cudaDeviceReset reloads the module; during capture the address from the
// last call outside capture is used (the lookup may load the module, which
// capture does not allow).
uint64_t* scratch_ptr(int dev, bool capturing, cudaError_t* err) {
  static std::mutex mu;
  static uint64_t* ptrs[64] = {nullptr};
  std::lock_guard<std::mutex> lock(mu);
  *err = cudaSuccess;
  if (dev < 0 || dev >= 64) {
    *err = cudaErrorInvalidDevice;
    return nullptr;
  }
  if (!capturing) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      *err = e;
      ptrs[dev] = nullptr;
      return nullptr;
    }
    ptrs[dev] = (uint64_t*)p;
  } else if (!ptrs[dev]) {
    *err = cudaErrorStreamCaptureUnsupported;
  }
  return ptrs[dev];
}

// exclusive scan of n u64 in place (out[n] = total): per-block sums, a scan
// of the sums in one block, then each block's scan from its offset
__device__ uint64_t na_block_scan(uint64_t v, uint64_t* total) {
  __shared__ uint64_t ws[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    uint64_t t = lane < nw ? ws[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(FULL, t, o);
      if (lane >= o) t += y;
    }
    if (lane < nw) ws[lane] = t;
  }
  __syncthreads();
  const uint64_t base = warp ? ws[warp - 1] : 0;
  if (total) *total = ws[(blockDim.x >> 5) - 1];
  __syncthreads();
  return base + x - v;
}

__global__ void k_na_scan_sums(const uint64_t* a, uint64_t n, uint64_t* bsum) {
  const uint64_t i0 = (uint64_t)blockIdx.x * NA_CH + (uint64_t)threadIdx.x * NA_PER;
  uint64_t s = 0;
  for (int k = 0; k < NA_PER; k++) s += i0 + k < n ? a[i0 + k] : 0;
  uint64_t tot;
  na_block_scan(s, &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_na_scan_top(uint64_t* bsum, uint64_t nb) {
  __shared__ uint64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint64_t c0 = 0; c0 < nb; c0 += blockDim.x) {
    const uint64_t i = c0 + threadIdx.x;
    uint64_t tot;
    const uint64_t ex = na_block_scan(i < nb ? bsum[i] : 0, &tot);
    if (i < nb) bsum[i] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) bsum[nb] = carry;
}

__global__ void k_na_scan_down(uint64_t* a, uint64_t n, const uint64_t* bsum) {
  const uint64_t i0 = (uint64_t)blockIdx.x * NA_CH + (uint64_t)threadIdx.x * NA_PER;
  uint64_t v[NA_PER], s = 0;
  for (int k = 0; k < NA_PER; k++) {
    v[k] = i0 + k < n ? a[i0 + k] : 0;
    s += v[k];
  }
  uint64_t ex = na_block_scan(s, nullptr) + bsum[blockIdx.x];
  for (int k = 0; k < NA_PER; k++) {
    if (i0 + k < n) a[i0 + k] = ex;
    ex += v[k];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) a[n] = bsum[gridDim.x];
}

__global__ void k_rs_count_static(const uint64_t* bits, uint64_t nbits, uint64_t nsb,
                                  uint64_t* dir, uint64_t* sbz) {
  const int lane = threadIdx.x & 31;
  const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t s = gw; s < nsb; s += nw) {
    const int64_t rem = (int64_t)nbits - (int64_t)(2048 * s + 64 * (uint64_t)lane);
    const int valid = rem <= 0 ? 0 : (rem >= 64 ? 64 : (int)rem);
    const uint64_t w = valid ? bits[32 * s + lane] : 0ull;
    const int z = valid - __popcll(w);
    int zi = z;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(FULL, zi, o);
      if (lane >= o) zi += y;
    }
    const uint64_t r1 = (uint64_t)__shfl_sync(FULL, zi, 7);
    const uint64_t r2 = (uint64_t)__shfl_sync(FULL, zi, 15);
    const uint64_t r3 = (uint64_t)__shfl_sync(FULL, zi, 23);
    if (lane == 0) dir[2 * s + 1] = (r1 << 16) | (r2 << 32) | (r3 << 48);
    if (lane == 31) sbz[s] = (uint64_t)zi;
  }
}

__global__ void k_rs_finish_static(uint64_t nsb, const uint64_t* sbx, uint64_t* dir) {
  const uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < nsb) dir[2 * s] = sbx[s];
  if (s == nsb) {
    dir[2 * nsb] = sbx[nsb];
    dir[2 * nsb + 1] = 0;
  }
}

__device__ __forceinline__ uint32_t sel64_static(uint64_t v, uint32_t r) {
  const uint32_t lo = (uint32_t)v, hi = (uint32_t)(v >> 32);
  const uint32_t pl = __popc(lo);
  if (r < pl) return __fns(lo, 0, (int)r + 1);
  return 32 + __fns(hi, 0, (int)(r - pl) + 1);
}

__device__ uint32_t find_in_sb_static(const uint64_t* bits, const uint64_t* dir, uint64_t s,
                                      int bv, uint32_t r) {
  const uint64_t rel = dir[2 * s + 1];
  int b = 3;
  for (; b > 0; b--) {
    const uint32_t z = (uint32_t)((rel >> (16 * b)) & 0xffffu);
    if ((bv ? 512u * b - z : z) <= r) break;
  }
  const uint32_t z = b ? (uint32_t)((rel >> (16 * b)) & 0xffffu) : 0u;
  r -= bv ? 512u * b - z : z;
  for (uint64_t w = 32 * s + 8 * b; w < 32 * s + 32; w++) {
    const uint64_t v = bits[w];
    const uint32_t c = bv ? __popcll(v) : 64 - __popcll(v);
    if (c > r) return (uint32_t)((w - 32 * s) * 64) + sel64_static(bv ? v : ~v, r);
    r -= c;
  }
  return 2047;
}

__global__ void k_rs_select_static(const uint64_t* bits, uint64_t nbits, uint64_t nsb,
                                   const uint64_t* dir, uint64_t* samp0, uint64_t* samp1) {
  const uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsb) return;
  const uint64_t zb = dir[2 * s], zs = dir[2 * s + 2] - zb;
  const uint64_t nvalid = nbits - 2048 * s < 2048 ? nbits - 2048 * s : 2048;
  const uint64_t ob = 2048 * s - zb, os = nvalid - zs;
  const uint64_t k0 = (zb + 4095) / 4096;
  if (4096 * k0 < zb + zs)
    samp0[k0] = 2048 * s + find_in_sb_static(bits, dir, s, 0, (uint32_t)(4096 * k0 - zb));
  const uint64_t k1 = (ob + 4095) / 4096;
  if (4096 * k1 < ob + os)
    samp1[k1] = 2048 * s + find_in_sb_static(bits, dir, s, 1, (uint32_t)(4096 * k1 - ob));
}

}  // namespace
}  // namespace wtk

using namespace wtk;

// One launch with its own return code: the error of this launch only (an
// error an earlier, unrelated call left pending is neither reported as this
// call's nor cleared).
template <class T>
struct same_type {
  using type = T;
};
template <typename... A>
static cudaError_t launch(void (*k)(A...), unsigned grid, unsigned block, cudaStream_t st,
                          typename same_type<A>::type... args) {
  void* pa[] = {(void*)&args...};
  const cudaError_t e = cudaLaunchKernel((const void*)k, dim3(grid), dim3(block), pa, 0, st);
  if (e == cudaSuccess) count_launch();
  return e;
}

extern "C" wt_status rs_dir_build_static(const uint64_t* d_bits, uint64_t nbits, uint64_t* d_dir,
                                         uint64_t* d_samp0, uint64_t* d_samp1,
                                         wt_stream stream) {
  if (nbits > NOALLOC_MAX_BITS) {
    fprintf(stderr, "rs_dir_build_static: %llu bits exceed the limit of %llu bits\n",
            (unsigned long long)nbits, (unsigned long long)NOALLOC_MAX_BITS);
    return WT_ERR_UNSUPPORTED;
  }
  if (!d_dir || (nbits && (!d_bits || !d_samp0 || !d_samp1))) return WT_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return WT_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return WT_ERR_CUDA;
  cudaError_t err;
  uint64_t* scr = scratch_ptr(dev, cap != cudaStreamCaptureStatusNone, &err);
  if (!scr) {
    fprintf(stderr, "rs_dir_build_static: no device address of the scratch array: %s\n",
            cudaGetErrorString(err));
    return WT_ERR_CUDA;
  }
  const uint64_t nsb = (nbits + 2047) / 2048;
  uint64_t* sbz = scr;                 // nsb + 1 entries, scanned in place
  uint64_t* bsum = scr + NOALLOC_MAX_SB + 1;
  // every scratch entry read below is written first by this call
  cudaError_t e = cudaSuccess;
  const uint64_t nb = (nsb + NA_CH - 1) / NA_CH;
  if (nsb) {
    e = launch(k_rs_count_static, (unsigned)((nsb * 32 + 255) / 256), 256u, st, d_bits, nbits,
               nsb, d_dir, sbz);
    if (e == cudaSuccess) e = launch(k_na_scan_sums, (unsigned)nb, (unsigned)NA_BT, st,
                                     sbz, nsb, bsum);
    if (e == cudaSuccess) e = launch(k_na_scan_top, 1u, (unsigned)NA_BT, st, bsum, nb);
    if (e == cudaSuccess) e = launch(k_na_scan_down, (unsigned)nb, (unsigned)NA_BT, st, sbz, nsb,
                                     bsum);
  } else {
    e = cudaMemsetAsync(sbz, 0, sizeof(uint64_t), st);
  }
  if (e == cudaSuccess) e = launch(k_rs_finish_static, (unsigned)((nsb + 1 + 255) / 256), 256u,
                                   st, nsb, sbz, d_dir);
  if (e == cudaSuccess && nsb)
    e = launch(k_rs_select_static, (unsigned)((nsb + 255) / 256), 256u, st, d_bits, nbits, nsb,
               d_dir, d_samp0, d_samp1);
  if (e != cudaSuccess) {
    cudaGetLastError();  // this call's own launch error, returned as the status
    fprintf(stderr, "rs_dir_build_static: %s\n", cudaGetErrorString(e));
    return WT_ERR_CUDA;
  }
  return WT_OK;
}
