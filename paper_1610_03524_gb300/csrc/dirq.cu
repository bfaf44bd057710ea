// dirq.cu -- rank/select directories on every level (Section 5) and the
// batched query kernels (access / rank / select, Section 2 definitions).
//
// Binary levels (Section 5.1, rank of 0 only, Jacobson-style two-level
// counts): one 16-byte record per 2048-bit superblock, {u64 zeros before the
// superblock, 4 x u16 zeros before each 512-bit block inside it}, plus a
// trailing record with the level total.  Select (Section 5.1, positions of
// every k-th bit kept, here k = 4096): the position of the occurrence with
// 0-based index 4096k of each bit value; a query starts at the sample and
// searches superblocks, blocks, words, then the bit inside the word.
// Digit levels of the 4-ary tree (Section 5.2, per-value counts): one
// 64-byte record per 1024 digits, {4 x u64 counts of each value before the
// superblock, 4 blocks x 4 values u16 counts inside it}; select samples per
// digit value (Section 5.2 generalized select: the position of every 4096th
// occurrence of each value), four regions of n/4096 + 1 per level.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "wt_host.h"
#include "wt_internal.cuh"

namespace wtk {

constexpr uint64_t NONE = ~0ull;

#define CK(x)                                                   \
  do {                                                          \
    cudaError_t e_ = (x);                                       \
    if (e_ != cudaSuccess) {                                    \
      fprintf(stderr, "wavelet: %s -> %s\n", #x, cudaGetErrorString(e_)); \
      return e_ == cudaErrorMemoryAllocation ? WT_ERR_NO_MEMORY : WT_ERR_CUDA; \
    }                                                           \
  } while (0)

// exclusive u64 scan from build.cu
wt_status scan_excl_u64_pub(const uint64_t* in, uint64_t* out, uint64_t n, uint64_t* scratch,
                            cudaStream_t st);
uint64_t scan_scratch_pub(uint64_t n);

// the level holding superblock g: last l with first[l] <= g (levels with no
// superblock share their first with the next level and are skipped)
__device__ __forceinline__ int find_level(const uint64_t* first, int nlev, uint64_t g) {
  int lo = 0, hi = nlev - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// r-th (0-based) set bit of v
__device__ __forceinline__ uint32_t sel64(uint64_t v, uint32_t r) {
  const uint32_t lo = (uint32_t)v, hi = (uint32_t)(v >> 32);
  const uint32_t pl = __popc(lo);
  if (r < pl) return __fns(lo, 0, (int)r + 1);
  return 32 + __fns(hi, 0, (int)(r - pl) + 1);
}

// ---------------------------------------------------------------------------
// binary directories
// ---------------------------------------------------------------------------
// One block covers DIR_SB_PER_BLOCK superblocks of one level (blk_first[l]:
// first block of level l), so the level is found once per block; each warp
// counts DIR_SB_PER_WARP superblocks with their words loaded together.
#ifndef WT_DIR_SB_PER_WARP
#define WT_DIR_SB_PER_WARP 8
#endif
constexpr int DIR_SB_PER_WARP = WT_DIR_SB_PER_WARP;
constexpr int DIR_SB_PER_BLOCK = 8 * DIR_SB_PER_WARP;  // 256 threads

// Up to DIR_SMALL levels: their first blocks, first superblocks and
// metadata ride in the kernel parameters, so a block finds its level without
// a dependent load (else the tables are searched in global memory).
constexpr int DIR_SMALL = 32;
struct DirLevels {
  int nlev;
  uint64_t blk_first[DIR_SMALL + 1];
  uint64_t sb_first[DIR_SMALL + 1];
  LevelMeta meta[DIR_SMALL];
};

template <bool SMALL>
__global__ void __launch_bounds__(256) k_dir_count(const uint64_t* bits, const LevelMeta* meta,
                                                   int nlev, const uint64_t* sb_first,
                                                   const uint64_t* blk_first, uint64_t* dir,
                                                   uint64_t* sbz, const __grid_constant__ DirLevels dl) {
  __shared__ LevelMeta sm;
  __shared__ uint64_t s_sb0, s_g0;
  LevelMeta m;
  uint64_t sb0, g0;
  if (SMALL) {
    int l = 0;
    while (l + 1 < dl.nlev && dl.blk_first[l + 1] <= blockIdx.x) l++;
    m = dl.meta[l];
    sb0 = (blockIdx.x - dl.blk_first[l]) * DIR_SB_PER_BLOCK;
    g0 = dl.sb_first[l];
  } else {
    if (threadIdx.x == 0) {
      const int l = find_level(blk_first, nlev, blockIdx.x);
      sm = meta[l];
      s_sb0 = (blockIdx.x - blk_first[l]) * DIR_SB_PER_BLOCK;
      s_g0 = sb_first[l];
    }
    __syncthreads();
    m = sm;
    sb0 = s_sb0;
    g0 = s_g0;
  }
  // two superblocks at a time: lanes 0-15 the first, 16-31 the second, each
  // lane two consecutive words (one 16-byte load where aligned)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int hl = lane & 15, half = lane >> 4;
  const uint64_t s0 = sb0 + (uint64_t)warp * DIR_SB_PER_WARP;
  const uint64_t* lb = bits + m.bit_off;
  const bool vec = (((uintptr_t)lb) & 15) == 0;
  constexpr int NP = DIR_SB_PER_WARP / 2;
  uint64_t w0[NP], w1[NP];
  int v0[NP], v1[NP];
#pragma unroll
  for (int u = 0; u < NP; u++) {
    const uint64_t s = s0 + 2 * u + half;
    const int64_t rem = (int64_t)m.n - (int64_t)(2048 * s + 128 * (uint64_t)hl);
    const bool live = s < m.nsb && rem > 0;
    v0[u] = !live ? 0 : (rem >= 64 ? 64 : (int)rem);
    v1[u] = (!live || rem <= 64) ? 0 : (rem >= 128 ? 64 : (int)(rem - 64));
    const uint64_t* p = lb + 32 * s + 2 * hl;
    // words past the last valid bit are not read (a caller bitvector may end there)
    if (v1[u] && vec) {
      const ulonglong2 q = __ldcs((const ulonglong2*)p);
      w0[u] = q.x;
      w1[u] = q.y;
    } else {
      w0[u] = v0[u] ? __ldcs(p) : 0ull;
      w1[u] = v1[u] ? __ldcs(p + 1) : 0ull;
    }
  }
#pragma unroll
  for (int u = 0; u < NP; u++) {
    const uint64_t s = s0 + 2 * u + half;
    const int z = v0[u] + v1[u] - __popcll(w0[u]) - __popcll(w1[u]);
    int zi = z;
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) {
      const int y = __shfl_up_sync(FULL, zi, o, 16);
      if (hl >= o) zi += y;
    }
    // zeros of 512-bit blocks 0, 1, 2 of the superblock: lanes 3, 7, 11 of its half
    const uint64_t r1 = (uint64_t)__shfl_sync(FULL, zi, 3, 16);
    const uint64_t r2 = (uint64_t)__shfl_sync(FULL, zi, 7, 16);
    const uint64_t r3 = (uint64_t)__shfl_sync(FULL, zi, 11, 16);
    if (s < m.nsb) {
      if (hl == 0) dir[m.dir_off + 2 * s + 1] = (r1 << 16) | (r2 << 32) | (r3 << 48);
      if (hl == 15) sbz[g0 + s] = (uint64_t)zi;
    }
  }
}

__global__ void k_dir_finish(const LevelMeta* meta, int nlev, const uint64_t* sb_first,
                             uint64_t total_sb, const uint64_t* sbx, uint64_t* dir,
                             uint64_t* zeros, int write_zeros) {
  const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < total_sb) {
    const int l = find_level(sb_first, nlev, g);
    const uint64_t s = g - sb_first[l];
    dir[meta[l].dir_off + 2 * s] = sbx[g] - sbx[sb_first[l]];
  } else if (g < total_sb + nlev) {
    const int l = (int)(g - total_sb);
    const LevelMeta m = meta[l];
    const uint64_t tot = sbx[sb_first[l + 1]] - sbx[sb_first[l]];
    dir[m.dir_off + 2 * m.nsb] = tot;
    dir[m.dir_off + 2 * m.nsb + 1] = 0;
    if (write_zeros) zeros[l] = tot;
  }
}

// position (inside superblock s, relative to its start) of the r-th
// (0-based) bit equal to bv
__device__ uint32_t find_in_sb(const uint64_t* lbits, const uint64_t* ldir, uint64_t s, int bv,
                               uint32_t r) {
  const uint64_t rel = ldir[2 * s + 1];
  int b = 3;
  for (; b > 0; b--) {
    const uint32_t z = (uint32_t)((rel >> (16 * b)) & 0xffffu);
    const uint32_t before = bv ? 512u * b - z : z;
    if (before <= r) break;
  }
  const uint32_t z = b ? (uint32_t)((rel >> (16 * b)) & 0xffffu) : 0u;
  r -= bv ? 512u * b - z : z;
  // the target lies in this superblock, so at most 32 words are visited
  for (uint64_t w = 32 * s + 8 * b; w < 32 * s + 32; w++) {
    const uint64_t v = lbits[w];
    const uint32_t c = bv ? __popcll(v) : 64 - __popcll(v);
    if (c > r) return (uint32_t)((w - 32 * s) * 64) + sel64(bv ? v : ~v, r);
    r -= c;
  }
  return 2047;
}

// The same for the sample kernel, with the target block's eight words loaded
// together (one round of loads instead of one per word visited); words at
// or past nw, the level's word count, are not read.
__device__ uint32_t find_in_sb_blk(const uint64_t* lbits, const uint64_t* ldir, uint64_t s,
                                   int bv, uint32_t r, uint64_t nw) {
  const uint64_t rel = ldir[2 * s + 1];
  int b = 3;
  for (; b > 0; b--) {
    const uint32_t z = (uint32_t)((rel >> (16 * b)) & 0xffffu);
    const uint32_t before = bv ? 512u * b - z : z;
    if (before <= r) break;
  }
  const uint32_t z = b ? (uint32_t)((rel >> (16 * b)) & 0xffffu) : 0u;
  r -= bv ? 512u * b - z : z;
  const uint64_t w0 = 32 * s + 8 * (uint64_t)b;
  uint64_t v[8];
#pragma unroll
  for (int i = 0; i < 8; i++) v[i] = w0 + i < nw ? lbits[w0 + i] : 0ull;
#pragma unroll
  for (int i = 0; i < 8; i++) {
    const uint32_t c = bv ? __popcll(v[i]) : 64 - __popcll(v[i]);
    if (c > r) return (uint32_t)((8 * b + i) * 64) + sel64(bv ? v[i] : ~v[i], r);
    r -= c;
  }
  return 2047;
}

template <bool SMALL>
__global__ void k_select_samples(const uint64_t* bits, const LevelMeta* meta, int nlev,
                                 const uint64_t* sb_first, uint64_t total_sb,
                                 const uint64_t* dir, uint64_t* samp,
                                 const __grid_constant__ DirLevels dl) {
  const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total_sb) return;
  LevelMeta m;
  uint64_t s;
  if (SMALL) {
    int l = 0;
    while (l + 1 < dl.nlev && dl.sb_first[l + 1] <= g) l++;
    m = dl.meta[l];
    s = g - dl.sb_first[l];
  } else {
    const int l = find_level(sb_first, nlev, g);
    m = meta[l];
    s = g - sb_first[l];
  }
  const uint64_t* ld = dir + m.dir_off;
  const uint64_t* lb = bits + m.bit_off;
  const uint64_t zb = ld[2 * s], ze = ld[2 * s + 2];
  const uint64_t zs = ze - zb;
  const uint64_t nvalid = std::min<uint64_t>(2048, m.n - 2048 * s);
  const uint64_t ob = 2048 * s - zb, os = nvalid - zs;
  const uint64_t nw = (m.n + 63) / 64;
  const uint64_t k0 = (zb + 4095) / 4096;
  if (4096 * k0 < zb + zs)
    samp[m.s0_off + k0] = 2048 * s + find_in_sb_blk(lb, ld, s, 0, (uint32_t)(4096 * k0 - zb), nw);
  const uint64_t k1 = (ob + 4095) / 4096;
  if (4096 * k1 < ob + os)
    samp[m.s1_off + k1] = 2048 * s + find_in_sb_blk(lb, ld, s, 1, (uint32_t)(4096 * k1 - ob), nw);
}

// ---------------------------------------------------------------------------
// digit-level (4-ary) directories
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t digit_match(uint64_t w, uint32_t d) {
  const uint64_t x = w ^ (0x5555555555555555ull * d);
  return ~(x | (x >> 1)) & 0x5555555555555555ull;
}

// The same counts, laid out like k_dir_count for up to DIR_SMALL levels:
// DIR_SB_PER_BLOCK superblocks of one level per block, two superblocks per
// warp step (each half-warp one: 16 lanes x two words = 1024 digits), 16-byte
// loads.  A lane holds 64 digits, so the 256-digit blocks end at lanes 3, 7,
// 11 of its half.
__global__ void __launch_bounds__(256) k_mdir_count_blk(const uint64_t* bits, uint64_t total_sb,
                                                        uint64_t* dir, uint64_t* sbz,
                                                        const __grid_constant__ DirLevels dl) {
  int l = 0;
  while (l + 1 < dl.nlev && dl.blk_first[l + 1] <= blockIdx.x) l++;
  const LevelMeta m = dl.meta[l];
  const uint64_t sb0 = (blockIdx.x - dl.blk_first[l]) * DIR_SB_PER_BLOCK;
  const uint64_t g0 = dl.sb_first[l];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int hl = lane & 15, half = lane >> 4;
  const uint64_t s0 = sb0 + (uint64_t)warp * DIR_SB_PER_WARP;
  const uint64_t* lb = bits + m.bit_off;
  const bool vec = (((uintptr_t)lb) & 15) == 0;
  constexpr int NP = DIR_SB_PER_WARP / 2;
  uint64_t w0[NP], w1[NP];
  int v0[NP], v1[NP];  // valid digits of the two words
#pragma unroll
  for (int u = 0; u < NP; u++) {
    const uint64_t s = s0 + 2 * u + half;
    const int64_t rem = (int64_t)m.n - (int64_t)(1024 * s + 64 * (uint64_t)hl);
    const bool live = s < m.nsb && rem > 0;
    v0[u] = !live ? 0 : (rem >= 32 ? 32 : (int)rem);
    v1[u] = (!live || rem <= 32) ? 0 : (rem >= 64 ? 32 : (int)(rem - 32));
    const uint64_t* p = lb + 32 * s + 2 * hl;
    if (v1[u] && vec) {
      const ulonglong2 q = __ldcs((const ulonglong2*)p);
      w0[u] = q.x;
      w1[u] = q.y;
    } else {
      w0[u] = v0[u] ? __ldcs(p) : 0ull;
      w1[u] = v1[u] ? __ldcs(p + 1) : 0ull;
    }
  }
#pragma unroll
  for (int u = 0; u < NP; u++) {
    const uint64_t s = s0 + 2 * u + half;
    const uint64_t vm0 = v0[u] >= 32 ? ~0ull : ((1ull << (2 * v0[u])) - 1ull);
    const uint64_t vm1 = v1[u] >= 32 ? ~0ull : ((1ull << (2 * v1[u])) - 1ull);
    uint64_t rec = 0;  // lane hl < 4: the four values' counts before block hl
#pragma unroll
    for (int d = 0; d < 4; d++) {
      int ci = __popcll(digit_match(w0[u], d) & vm0) + __popcll(digit_match(w1[u], d) & vm1);
#pragma unroll
      for (int o = 1; o < 16; o <<= 1) {
        const int y = __shfl_up_sync(FULL, ci, o, 16);
        if (hl >= o) ci += y;
      }
      const uint32_t r1 = (uint32_t)__shfl_sync(FULL, ci, 3, 16);
      const uint32_t r2 = (uint32_t)__shfl_sync(FULL, ci, 7, 16);
      const uint32_t r3 = (uint32_t)__shfl_sync(FULL, ci, 11, 16);
      const uint32_t rb = hl == 1 ? r1 : (hl == 2 ? r2 : (hl == 3 ? r3 : 0u));
      rec |= (uint64_t)rb << (16 * d);
      if (hl == 15 && s < m.nsb) sbz[(uint64_t)d * total_sb + g0 + s] = (uint64_t)ci;
    }
    if (hl < 4 && s < m.nsb) dir[m.dir_off + 8 * s + 4 + hl] = rec;
  }
}

__global__ void k_mdir_count(const uint64_t* bits, const LevelMeta* meta, int nlev,
                             const uint64_t* sb_first, uint64_t total_sb, uint64_t* dir,
                             uint64_t* sbz /* 4 x total_sb */) {
  const int lane = threadIdx.x & 31;
  const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t g = gw; g < total_sb; g += nw) {
    const int l = find_level(sb_first, nlev, g);
    const LevelMeta m = meta[l];
    const uint64_t s = g - sb_first[l];
    const int64_t rem = (int64_t)m.n - (int64_t)(1024 * s + 32 * (uint64_t)lane);
    const int valid = rem <= 0 ? 0 : (rem >= 32 ? 32 : (int)rem);
    const uint64_t w = valid ? bits[m.bit_off + 32 * s + lane] : 0ull;
    const uint64_t vm = valid == 32 ? ~0ull : ((1ull << (2 * valid)) - 1ull);
    uint64_t packed[4];
#pragma unroll
    for (int d = 0; d < 4; d++) {
      int c = __popcll(digit_match(w, d) & vm);
      int ci = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, ci, o);
        if (lane >= o) ci += y;
      }
      const uint64_t r1 = (uint64_t)__shfl_sync(FULL, ci, 7);
      const uint64_t r2 = (uint64_t)__shfl_sync(FULL, ci, 15);
      const uint64_t r3 = (uint64_t)__shfl_sync(FULL, ci, 23);
      packed[d] = (r1 << 16) | (r2 << 32) | (r3 << 48);  // rel of blocks 1..3 for value d
      if (lane == 31) sbz[(uint64_t)d * total_sb + g] = (uint64_t)ci;
    }
    if (lane < 4) {
      // record word 4+b holds the four values' counts of block b
      const int b = lane;
      uint64_t v = 0;
#pragma unroll
      for (int d = 0; d < 4; d++) v |= ((packed[d] >> (16 * b)) & 0xffffull) << (16 * d);
      dir[m.dir_off + 8 * s + 4 + b] = v;
    }
  }
}

__global__ void k_mdir_finish(const LevelMeta* meta, int nlev, const uint64_t* sb_first,
                              uint64_t total_sb, const uint64_t* sbx /* 4 x (total_sb+1) */,
                              uint64_t* dir) {
  const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < total_sb) {
    const int l = find_level(sb_first, nlev, g);
    const uint64_t s = g - sb_first[l];
    for (int d = 0; d < 4; d++) {
      const uint64_t* x = sbx + (uint64_t)d * (total_sb + 1);
      dir[meta[l].dir_off + 8 * s + d] = x[g] - x[sb_first[l]];
    }
  } else if (g < total_sb + nlev) {
    const int l = (int)(g - total_sb);
    const LevelMeta m = meta[l];
    for (int d = 0; d < 4; d++) {
      const uint64_t* x = sbx + (uint64_t)d * (total_sb + 1);
      dir[m.dir_off + 8 * m.nsb + d] = x[sb_first[l + 1]] - x[sb_first[l]];
      dir[m.dir_off + 8 * m.nsb + 4 + d] = 0;
    }
  }
}

// position (inside digit superblock s, relative to its start) of the r-th
// (0-based) occurrence of digit value d; the occurrence lies in s
__device__ uint32_t find_in_dsb(const uint64_t* lbits, const uint64_t* ldir, uint64_t s, uint32_t d,
                                uint32_t r) {
  int b = 3;
  for (; b > 0; b--)
    if (((ldir[8 * s + 4 + b] >> (16 * d)) & 0xffffull) <= r) break;
  r -= b ? (uint32_t)((ldir[8 * s + 4 + b] >> (16 * d)) & 0xffffull) : 0u;
  for (uint64_t w = 32 * s + 8 * b; w < 32 * s + 32; w++) {
    const uint64_t m = digit_match(lbits[w], d);
    const uint32_t c = __popcll(m);
    if (c > r) return (uint32_t)((w - 32 * s) * 32 + sel64(m, r) / 2);
    r -= c;
  }
  return 1023;
}

// every 4096th occurrence of each digit value: one thread per superblock
// (a superblock of 1024 digits holds at most one sample per value)
__global__ void k_mdigit_samples(const uint64_t* bits, const LevelMeta* meta, int nlev,
                                 const uint64_t* sb_first, uint64_t total_sb,
                                 const uint64_t* dir, uint64_t* samp) {
  const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total_sb) return;
  const int l = find_level(sb_first, nlev, g);
  const LevelMeta m = meta[l];
  const uint64_t s = g - sb_first[l];
  const uint64_t* ld = dir + m.dir_off;
  const uint64_t* lb = bits + m.bit_off;
  const uint64_t cap = m.n / 4096 + 1;
  for (uint32_t d = 0; d < 4; d++) {
    const uint64_t before = ld[8 * s + d], in = ld[8 * (s + 1) + d] - before;
    const uint64_t k = (before + 4095) / 4096;
    if (4096 * k < before + in)
      samp[m.s0_off + d * cap + k] = 1024 * s + find_in_dsb(lb, ld, s, d, (uint32_t)(4096 * k - before));
  }
}

wt_status upload_meta(wt_struct* h) {
  const size_t nb = std::max<size_t>(h->meta.size(), 1) * sizeof(LevelMeta);
  if (!h->d_meta) CK(dmalloc((void**)&h->d_meta, nb, h->stream));
  if (!h->meta.empty()) return upload(h->d_meta, h->meta.data(), h->meta.size() * sizeof(LevelMeta), h->stream);
  return WT_OK;
}

// Binary directories and select samples of nlev levels described by d_meta
// (offsets relative to bits / dir / samp); sb_first: first superblock of each
// level in one numbering, its first nlev + 1 entries used.  write_zeros: also store each
// level's zero count in zeros[l].
wt_status dir_build_levels(const uint64_t* bits, const LevelMeta* d_meta, uint32_t nlev,
                           const std::vector<uint64_t>& sb_first, uint64_t* dir, uint64_t* samp,
                           uint64_t* zeros, int write_zeros, cudaStream_t st,
                           const LevelMeta* h_meta) {
  if (nlev == 0) return WT_OK;
  const uint64_t total_sb = sb_first[nlev];
  // blocks of the counting kernel: DIR_SB_PER_BLOCK superblocks of one level each
  std::vector<uint64_t> firsts(2 * ((size_t)nlev + 1), 0);
  std::copy(sb_first.begin(), sb_first.begin() + nlev + 1, firsts.begin());
  uint64_t* blk_first = firsts.data() + nlev + 1;
  for (uint32_t l = 0; l < nlev; l++) {
    const uint64_t nsb = sb_first[l + 1] - sb_first[l];
    blk_first[l + 1] = blk_first[l] + (nsb + DIR_SB_PER_BLOCK - 1) / DIR_SB_PER_BLOCK;
  }
  const uint64_t nblk = blk_first[nlev];
  Work wk{st, {}};
  uint64_t *d_first, *sbz, *sbx, *scr;
  TRY(wk.get(&d_first, 2 * ((size_t)nlev + 1)));
  TRY(wk.get(&sbz, std::max<uint64_t>(total_sb, 1)));
  TRY(wk.get(&sbx, total_sb + 1));
  TRY(wk.get(&scr, scan_scratch_pub(total_sb)));
  TRY(upload(d_first, firsts.data(), firsts.size() * 8, st));
  const unsigned fgrid = (unsigned)((total_sb + nlev + 255) / 256);
  // few levels with host metadata: the level tables go in the parameters
  const bool small = h_meta && nlev <= (uint32_t)DIR_SMALL;
  DirLevels dl;
  memset(&dl, 0, sizeof(dl));
  if (small) {
    dl.nlev = (int)nlev;
    for (uint32_t l = 0; l <= nlev; l++) {
      dl.blk_first[l] = blk_first[l];
      dl.sb_first[l] = sb_first[l];
    }
    for (uint32_t l = 0; l < nlev; l++) dl.meta[l] = h_meta[l];
  }
  if (total_sb) {
    if (small)
      k_dir_count<true><<<(unsigned)nblk, 256, 0, st>>>(bits, d_meta, (int)nlev, d_first,
                                                       d_first + nlev + 1, dir, sbz, dl);
    else
      k_dir_count<false><<<(unsigned)nblk, 256, 0, st>>>(bits, d_meta, (int)nlev, d_first,
                                                        d_first + nlev + 1, dir, sbz, dl);
    count_launch();
  }
  wt_status s = scan_excl_u64_pub(sbz, sbx, total_sb, scr, st);
  if (s == WT_OK) {
    k_dir_finish<<<fgrid, 256, 0, st>>>(d_meta, (int)nlev, d_first, total_sb, sbx, dir, zeros,
                                        write_zeros);
    count_launch();
    if (total_sb) {
      if (small)
        k_select_samples<true><<<(unsigned)((total_sb + 255) / 256), 256, 0, st>>>(
            bits, d_meta, (int)nlev, d_first, total_sb, dir, samp, dl);
      else
        k_select_samples<false><<<(unsigned)((total_sb + 255) / 256), 256, 0, st>>>(
            bits, d_meta, (int)nlev, d_first, total_sb, dir, samp, dl);
      count_launch();
    }
  }
  cudaError_t e = cudaGetLastError();
  if (s != WT_OK) return s;
  return e == cudaSuccess ? WT_OK : WT_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// constant-time select directory (after Clark, Section 5.1 select)
// ---------------------------------------------------------------------------
constexpr uint64_t CK_HUGE_MIN = 1ull << 32;    // range length that keeps all positions
constexpr uint64_t CK_SPARSE_MIN = 1ull << 16;  // sub-range length that keeps all offsets

// occurrences of value b before superblock s of a level: bit values of a
// binary level (2048-bit superblocks), digit values of a digit level (1024)
template <bool DIG>
__device__ __forceinline__ uint64_t occ_before(const uint64_t* ldir, int b, uint64_t s) {
  if (DIG) return ldir[8 * s + b];
  const uint64_t z = ldir[2 * s];
  return b ? 2048 * s - z : z;
}

// position of occurrence q of value b, known to lie in superblocks [lo, hi]
// of the level (q >= occurrences before lo)
template <bool DIG>
__device__ uint64_t dir_select(const uint64_t* lbits, const uint64_t* ldir, int b, uint64_t q,
                               uint64_t lo, uint64_t hi) {
  while (lo < hi) {
    const uint64_t mid = (lo + hi + 1) >> 1;
    if (occ_before<DIG>(ldir, b, mid) <= q) lo = mid;
    else hi = mid - 1;
  }
  const uint32_t r = (uint32_t)(q - occ_before<DIG>(ldir, b, lo));
  if (DIG) return 1024 * lo + find_in_dsb(lbits, ldir, lo, (uint32_t)b, r);
  return 2048 * lo + find_in_sb(lbits, ldir, lo, b, r);
}

// one (level, bit or digit value) of the directory build
struct CkSeg {
  uint64_t g0;        // its first range in the global numbering
  uint64_t cnt;       // occurrences
  uint64_t bit_off, dir_off, samp_off, n, nsb;
  int b;
};

__device__ __forceinline__ uint32_t ck_seg_of(const CkSeg* segs, uint32_t nseg, uint64_t g) {
  uint32_t lo = 0, hi = nseg - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (segs[mid].g0 <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// per range: kind, sub-sample offsets, mask of long sub-ranges
template <bool DIG>
__global__ void k_ck_ranges(const uint64_t* bits, const uint64_t* dir, const uint64_t* samp,
                            const CkSeg* segs, uint32_t nseg, uint64_t G, uint32_t* sub,
                            uint64_t* mask_or_huge, uint64_t* nh, uint64_t* ns) {
  const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G) return;
  const CkSeg sg = segs[ck_seg_of(segs, nseg, g)];
  const uint64_t k = g - sg.g0, R = (sg.cnt + 4095) / 4096;
  const uint64_t* lbits = bits + sg.bit_off;
  const uint64_t* ldir = dir + sg.dir_off;
  const uint64_t* ls = samp + sg.samp_off;
  const uint64_t S1 = ls[k];
  const uint64_t e = (k + 1 < R) ? ls[k + 1] : sg.n;
  const uint64_t M = (sg.cnt + 255) / 256;
  const bool huge = e - S1 >= CK_HUGE_MIN;
  uint32_t mask = 0;
  uint64_t prev = S1;  // start of sub-range i
  constexpr int SBSH = DIG ? 10 : 11;
  const uint64_t lo_sb = S1 >> SBSH, hi_sb = (e - 1) >> SBSH;
  for (int i = 0; i < 16; i++) {
    const uint64_t m = 16 * k + i;
    uint64_t start = 0;
    if (!huge && m < M) start = i == 0 ? S1 : dir_select<DIG>(lbits, ldir, sg.b, 256 * m, lo_sb, hi_sb);
    sub[16 * g + i] = huge ? 0u : (m < M ? (uint32_t)(start - S1) : 0xffffffffu);
    if (!huge && i > 0 && m - 1 < M && m < M && start - prev >= CK_SPARSE_MIN) mask |= 1u << (i - 1);
    if (!huge && m < M) prev = start;
    if (!huge && m < M && (i == 15 || m + 1 >= M) && e - start >= CK_SPARSE_MIN) mask |= 1u << i;
  }
  mask_or_huge[g] = huge ? (1ull << 63) : (uint64_t)mask;
  nh[g] = huge ? 1 : 0;
  ns[g] = huge ? 0 : (uint64_t)__popc(mask);
}

// descriptors, numbered inside their (level, bit value)
__global__ void k_ck_desc(const CkSeg* segs, uint32_t nseg, uint64_t G, const uint64_t* kind,
                          const uint64_t* gh, const uint64_t* gs, uint64_t* desc) {
  const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G) return;
  const CkSeg sg = segs[ck_seg_of(segs, nseg, g)];
  const uint64_t kd = kind[g];
  if (kd >> 63) desc[g] = (1ull << 63) | (4096 * (gh[g] - gh[sg.g0]));
  else desc[g] = (gs[g] - gs[sg.g0]) | (kd << 40);
}

// explicit answers: one block per range that keeps any
template <bool DIG>
__global__ void k_ck_fill(const uint64_t* bits, const uint64_t* dir, const uint64_t* samp,
                          const CkSeg* segs, uint32_t nseg, uint64_t G, const uint64_t* kind,
                          const uint64_t* gh, const uint64_t* gs, const uint32_t* sub,
                          uint64_t* huge_all, uint32_t* sparse_all) {
  for (uint64_t g = blockIdx.x; g < G; g += gridDim.x) {
    const uint64_t kd = kind[g];
    if (kd == 0) continue;
    const CkSeg sg = segs[ck_seg_of(segs, nseg, g)];
    const uint64_t k = g - sg.g0, R = (sg.cnt + 4095) / 4096;
    const uint64_t* lbits = bits + sg.bit_off;
    const uint64_t* ldir = dir + sg.dir_off;
    const uint64_t S1 = samp[sg.samp_off + k];
    const uint64_t e = (k + 1 < R) ? samp[sg.samp_off + k + 1] : sg.n;
    constexpr int SBSH = DIG ? 10 : 11;
    const uint64_t lo_sb = S1 >> SBSH, hi_sb = (e - 1) >> SBSH;
    if (kd >> 63) {
      for (uint32_t j = threadIdx.x; j < 4096; j += blockDim.x) {
        const uint64_t q = 4096 * k + j;
        huge_all[4096 * gh[g] + j] =
            q < sg.cnt ? dir_select<DIG>(lbits, ldir, sg.b, q, lo_sb, hi_sb) : ~0ull;
      }
    } else {
      uint32_t mask = (uint32_t)kd;
      uint64_t s = gs[g];
      while (mask) {
        const int i = __ffs(mask) - 1;
        mask &= mask - 1;
        for (uint32_t j = threadIdx.x; j < 256; j += blockDim.x) {
          const uint64_t q = 4096 * k + 256 * i + j;
          sparse_all[256 * s + j] =
              q < sg.cnt ? (uint32_t)(dir_select<DIG>(lbits, ldir, sg.b, q, lo_sb, hi_sb) - S1)
                         : 0xffffffffu;
        }
        s++;
      }
    }
  }
}

__global__ void k_gather_u64(const uint64_t* src, const uint64_t* idx, uint64_t n, uint64_t* out) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = src[idx[i]];
}

// dig: digit levels (4 values; occurrence counts from the directory's
// trailing records), else binary levels (2 values; counts from the zeros)
static wt_status build_clark(wt_struct* h) {
  cudaStream_t st = h->stream;
  const uint32_t nlev = h->levels;
  const bool dig = h->bpe == 2;
  const int NV = dig ? 4 : 2;
  // occurrence counts of every value on every level, on the host
  std::vector<uint64_t> occ((size_t)NV * nlev, 0);
  if (nlev) {
    if (dig) {
      std::vector<uint64_t> idx(occ.size());
      for (uint32_t l = 0; l < nlev; l++)
        for (int d = 0; d < 4; d++) idx[4 * l + d] = h->meta[l].dir_off + 8 * h->meta[l].nsb + d;
      Work wk0{st, {}};
      uint64_t *d_idx, *d_got;
      TRY(wk0.get(&d_idx, idx.size()));
      TRY(wk0.get(&d_got, idx.size()));
      TRY(upload(d_idx, idx.data(), idx.size() * 8, st));
      k_gather_u64<<<(unsigned)((idx.size() + 255) / 256), 256, 0, st>>>(h->d_dir, d_idx,
                                                                         idx.size(), d_got);
      count_launch();
      CK(cudaMemcpyAsync(occ.data(), d_got, occ.size() * 8, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
    } else {
      std::vector<uint64_t> zeros(nlev, 0);
      CK(cudaMemcpyAsync(zeros.data(), h->d_zeros, nlev * 8, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      for (uint32_t l = 0; l < nlev; l++) {
        occ[2 * l] = zeros[l];
        occ[2 * l + 1] = h->meta[l].n - zeros[l];
      }
    }
  }
  std::vector<CkSeg> segs;
  h->cmeta.assign(nlev, ClarkMeta{});
  uint64_t G = 0;
  for (uint32_t l = 0; l < nlev; l++) {
    const LevelMeta& m = h->meta[l];
    for (int b = 0; b < NV; b++) {
      CkSeg sg;
      sg.g0 = G;
      sg.cnt = occ[(size_t)NV * l + b];
      sg.bit_off = m.bit_off;
      sg.dir_off = m.dir_off;
      sg.samp_off = dig ? m.s0_off + (uint64_t)b * (m.n / 4096 + 1) : (b ? m.s1_off : m.s0_off);
      sg.n = m.n;
      sg.nsb = m.nsb;
      sg.b = b;
      const uint64_t R = (sg.cnt + 4095) / 4096;
      h->cmeta[l].nr[b] = R;
      h->cmeta[l].desc[b] = G;
      h->cmeta[l].sub[b] = 16 * G;
      if (R) segs.push_back(sg);
      G += R;
    }
  }
  const uint32_t nseg = (uint32_t)segs.size();
  Work wk{st, {}};
  uint64_t *d_kind, *d_nh, *d_ns, *d_gh, *d_gs, *scr;
  CkSeg* d_segs;
  uint32_t* d_sub;
  TRY(wk.get(&d_sub, std::max<uint64_t>(16 * G, 1)));
  TRY(wk.get(&d_kind, std::max<uint64_t>(G, 1)));
  TRY(wk.get(&d_nh, std::max<uint64_t>(G, 1)));
  TRY(wk.get(&d_ns, std::max<uint64_t>(G, 1)));
  TRY(wk.get(&d_gh, G + 1));
  TRY(wk.get(&d_gs, G + 1));
  TRY(wk.get(&scr, scan_scratch_pub(G)));
  TRY(wk.get(&d_segs, std::max<uint32_t>(nseg, 1)));
  if (nseg) TRY(upload(d_segs, segs.data(), nseg * sizeof(CkSeg), st));
  const unsigned gg = (unsigned)((G + 255) / 256);
  if (G) {
    if (dig)
      k_ck_ranges<true><<<gg, 256, 0, st>>>(h->d_bits_ro, h->d_dir, h->d_samp, d_segs, nseg, G,
                                            d_sub, d_kind, d_nh, d_ns);
    else
      k_ck_ranges<false><<<gg, 256, 0, st>>>(h->d_bits_ro, h->d_dir, h->d_samp, d_segs, nseg, G,
                                             d_sub, d_kind, d_nh, d_ns);
    count_launch();
  }
  wt_status s = scan_excl_u64_pub(d_nh, d_gh, G, scr, st);
  if (s == WT_OK) s = scan_excl_u64_pub(d_ns, d_gs, G, scr, st);
  uint64_t tot[2] = {0, 0};
  if (s == WT_OK) {
    CK(cudaMemcpyAsync(&tot[0], d_gh + G, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&tot[1], d_gs + G, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  const uint64_t H = tot[0], S = tot[1];
  if (s == WT_OK) {
    CK(dmalloc((void**)&h->d_ck64, std::max<uint64_t>(G + 4096 * H, 1) * 8, st));
    CK(dmalloc((void**)&h->d_ck32, std::max<uint64_t>(16 * G + 256 * S, 1) * 4, st));
    if (G) {
      CK(cudaMemcpyAsync(h->d_ck32, d_sub, 16 * G * 4, cudaMemcpyDeviceToDevice, st));
      k_ck_desc<<<gg, 256, 0, st>>>(d_segs, nseg, G, d_kind, d_gh, d_gs, h->d_ck64);
      count_launch();
      const unsigned fg = (unsigned)std::min<uint64_t>(G, (uint64_t)num_sms() * 16);
      if (dig)
        k_ck_fill<true><<<fg, 256, 0, st>>>(h->d_bits_ro, h->d_dir, h->d_samp, d_segs, nseg, G,
                                            d_kind, d_gh, d_gs, d_sub, h->d_ck64 + G,
                                            h->d_ck32 + 16 * G);
      else
        k_ck_fill<false><<<fg, 256, 0, st>>>(h->d_bits_ro, h->d_dir, h->d_samp, d_segs, nseg, G,
                                             d_kind, d_gh, d_gs, d_sub, h->d_ck64 + G,
                                             h->d_ck32 + 16 * G);
      count_launch();
    }
    // per (level, value): the scans at its first and one-past-last range
    const size_t nv = (size_t)NV * nlev;
    std::vector<uint64_t> idx(2 * nv, 0);
    for (uint32_t l = 0; l < nlev; l++)
      for (int b = 0; b < NV; b++) {
        idx[2 * (NV * l + b)] = h->cmeta[l].desc[b];
        idx[2 * (NV * l + b) + 1] = h->cmeta[l].desc[b] + h->cmeta[l].nr[b];
      }
    std::vector<uint64_t> both(2 * idx.size(), 0);
    if (nlev) {
      uint64_t *d_idx, *d_got;
      TRY(wk.get(&d_idx, idx.size()));
      TRY(wk.get(&d_got, both.size()));
      TRY(upload(d_idx, idx.data(), idx.size() * 8, st));
      k_gather_u64<<<(unsigned)((idx.size() + 255) / 256), 256, 0, st>>>(d_gh, d_idx, idx.size(), d_got);
      count_launch();
      k_gather_u64<<<(unsigned)((idx.size() + 255) / 256), 256, 0, st>>>(d_gs, d_idx, idx.size(),
                                                                         d_got + idx.size());
      count_launch();
      CK(cudaMemcpyAsync(both.data(), d_got, both.size() * 8, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
    }
    for (uint32_t l = 0; l < nlev; l++)
      for (int b = 0; b < NV; b++) {
        const size_t i = 2 * ((size_t)NV * l + b);
        ClarkMeta& cm = h->cmeta[l];
        cm.nh[b] = both[i + 1] - both[i];
        cm.ns[b] = both[idx.size() + i + 1] - both[idx.size() + i];
        cm.huge[b] = G + 4096 * both[i];
        cm.sparse[b] = 16 * G + 256 * both[idx.size() + i];
      }
    CK(dmalloc((void**)&h->d_cmeta, std::max<uint32_t>(nlev, 1) * sizeof(ClarkMeta), st));
    if (nlev)
      CK(cudaMemcpyAsync(h->d_cmeta, h->cmeta.data(), nlev * sizeof(ClarkMeta),
                         cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));  // host vectors above are pageable and local
  }
  cudaError_t e = cudaGetLastError();
  if (s != WT_OK) return s;
  return e == cudaSuccess ? WT_OK : WT_ERR_CUDA;
}

wt_status build_directories(wt_struct* h) {
  cudaStream_t st = h->stream;
  const uint32_t nlev = h->levels;
  const bool dig = h->bpe == 2;
  const uint64_t sbsz = dig ? 1024 : 2048;
  const uint64_t rec = dig ? 8 : 2;
  // select samples: per level one region of n/4096 + 1 per value (2 bit
  // values, or 4 digit values)
  const uint32_t NV = dig ? 4 : 2;
  h->meta.assign(nlev, LevelMeta{});
  h->dir_off.assign(nlev + 1, 0);
  h->samp_off.assign(NV * nlev + 1, 0);
  std::vector<uint64_t> sb_first(nlev + 1, 0);
  for (uint32_t l = 0; l < nlev; l++) {
    LevelMeta& m = h->meta[l];
    m.bit_off = h->level_off[l];
    m.n = h->level_len[l];
    m.nsb = (m.n + sbsz - 1) / sbsz;
    m.dir_off = h->dir_off[l];
    h->dir_off[l + 1] = h->dir_off[l] + rec * (m.nsb + 1);
    sb_first[l + 1] = sb_first[l] + m.nsb;
    const uint64_t cap = m.n / 4096 + 1;
    for (uint32_t v = 0; v < NV; v++) h->samp_off[NV * l + v + 1] = h->samp_off[NV * l + v] + cap;
    m.s0_off = h->samp_off[NV * l];
    m.s1_off = h->samp_off[NV * l + 1];
  }
  const uint64_t total_sb = sb_first[nlev];
  CK(dmalloc((void**)&h->d_dir, std::max<uint64_t>(h->dir_off[nlev], 1) * 8, st));
  CK(dmalloc((void**)&h->d_samp, std::max<uint64_t>(h->samp_off[NV * nlev], 1) * 8, st));
  wt_status s = upload_meta(h);
  if (s != WT_OK) return s;
  if (nlev == 0) return WT_OK;
  if (!dig) {
    s = dir_build_levels(h->d_bits_ro, h->d_meta, nlev, sb_first, h->d_dir, h->d_samp,
                         h->d_zeros, h->kind == WT_KIND_RS ? 1 : 0, st, h->meta.data());
    if (s == WT_OK && (h->flags & WT_FLAG_SELECT_O1)) s = build_clark(h);
    return s;
  }
  Work wk{st, {}};
  uint64_t *d_first, *sbz, *sbx, *scr;
  TRY(wk.get(&d_first, nlev + 1));
  TRY(wk.get(&sbz, std::max<uint64_t>(total_sb, 1) * 4));
  TRY(wk.get(&sbx, (total_sb + 1) * 4));
  TRY(wk.get(&scr, scan_scratch_pub(total_sb)));
  TRY(upload(d_first, sb_first.data(), (nlev + 1) * 8, st));
  const unsigned fgrid = (unsigned)((total_sb + nlev + 255) / 256);
  if (total_sb && nlev <= (uint32_t)DIR_SMALL) {
    // blocks of DIR_SB_PER_BLOCK superblocks of one level, the level tables
    // in the parameters
    DirLevels dl;
    memset(&dl, 0, sizeof(dl));
    dl.nlev = (int)nlev;
    for (uint32_t l = 0; l < nlev; l++) {
      dl.blk_first[l + 1] =
          dl.blk_first[l] + (h->meta[l].nsb + DIR_SB_PER_BLOCK - 1) / DIR_SB_PER_BLOCK;
      dl.sb_first[l + 1] = sb_first[l + 1];
      dl.meta[l] = h->meta[l];
    }
    k_mdir_count_blk<<<(unsigned)dl.blk_first[nlev], 256, 0, st>>>(h->d_bits_ro, total_sb,
                                                                  h->d_dir, sbz, dl);
    count_launch();
  } else if (total_sb) {
    // one warp per superblock: enough loads in flight to stream the bitmaps
    const unsigned cgrid = (unsigned)std::min<uint64_t>((total_sb * 32 + 255) / 256 + 1, 1u << 24);
    k_mdir_count<<<cgrid, 256, 0, st>>>(h->d_bits_ro, h->d_meta, nlev, d_first, total_sb,
                                        h->d_dir, sbz);
    count_launch();
  }
  for (int d = 0; d < 4 && s == WT_OK; d++)
    s = scan_excl_u64_pub(sbz + (uint64_t)d * total_sb, sbx + (uint64_t)d * (total_sb + 1),
                          total_sb, scr, st);
  if (s == WT_OK) {
    k_mdir_finish<<<fgrid, 256, 0, st>>>(h->d_meta, nlev, d_first, total_sb, sbx, h->d_dir);
    count_launch();
    if (total_sb) {
      k_mdigit_samples<<<(unsigned)((total_sb + 255) / 256), 256, 0, st>>>(
          h->d_bits_ro, h->d_meta, nlev, d_first, total_sb, h->d_dir, h->d_samp);
      count_launch();
    }
  }
  cudaError_t e = cudaGetLastError();
  if (s != WT_OK) return s;
  if (e != cudaSuccess) return WT_ERR_CUDA;
  if (h->flags & WT_FLAG_SELECT_O1) return build_clark(h);
  return WT_OK;
}

// ---------------------------------------------------------------------------
// queries
// ---------------------------------------------------------------------------
struct QStruct {
  int kind;
  uint64_t n;
  uint32_t sigma;
  int L;        // binary levels (HUFF: max code length)
  int levels;   // output levels
  const uint64_t* bits;
  const uint64_t* dir;
  const uint64_t* samp;
  const LevelMeta* meta;
  const uint64_t* zeros;
  HuffQuery hq;
  const ClarkMeta* cmeta;  // constant-time select directory, or null
  const uint64_t* ck64;
  const uint32_t* ck32;
};

struct BinLevel {
  const uint64_t* bits;
  const uint64_t* dir;
  const uint64_t* s0;
  const uint64_t* s1;
  uint64_t n, nsb, zeros;
  const ClarkMeta* cm;
  const uint64_t* ck64;
  const uint32_t* ck32;
};

__device__ __forceinline__ BinLevel bin_level(const QStruct& S, int l) {
  const LevelMeta m = S.meta[l];
  BinLevel v;
  v.bits = S.bits + m.bit_off;
  v.dir = S.dir + m.dir_off;
  v.s0 = S.samp + m.s0_off;
  v.s1 = S.samp + m.s1_off;
  v.n = m.n;
  v.nsb = m.nsb;
  v.zeros = S.zeros[l];
  v.cm = S.cmeta ? S.cmeta + l : nullptr;
  v.ck64 = S.ck64;
  v.ck32 = S.ck32;
  return v;
}

__device__ __forceinline__ int get_bit(const BinLevel& v, uint64_t i) {
  return (int)((v.bits[i >> 6] >> (i & 63)) & 1ull);
}

// zeros in [0, x), x <= n
__device__ uint64_t rank0(const BinLevel& v, uint64_t x) {
  const uint64_t s = x >> 11;
  const uint32_t b = (uint32_t)((x >> 9) & 3);
  uint64_t r = v.dir[2 * s] + ((v.dir[2 * s + 1] >> (16 * b)) & 0xffffull);
  const uint64_t wend = x >> 6;
  for (uint64_t w = 32 * s + 8 * b; w < wend; w++) r += 64 - __popcll(v.bits[w]);
  const uint32_t rem = (uint32_t)(x & 63);
  if (rem) r += rem - __popcll(v.bits[wend] & ((1ull << rem) - 1ull));
  return r;
}
__device__ __forceinline__ uint64_t rank1(const BinLevel& v, uint64_t x) { return x - rank0(v, x); }

// position of the k-th (0-based) bit equal to bv; k < count
__device__ uint64_t select_b(const BinLevel& v, int bv, uint64_t k) {
  const uint64_t* samp = bv ? v.s1 : v.s0;
  if (v.cm) {
    // constant-time directory: the range's descriptor gives the stored
    // answer, or a sub-range shorter than 2^16 bits to search
    const uint64_t kk = k >> 12;
    const uint64_t d = v.ck64[v.cm->desc[bv] + kk];
    if (d >> 63) return v.ck64[v.cm->huge[bv] + (d & ((1ull << 63) - 1)) + (k & 4095)];
    const uint32_t mask = (uint32_t)((d >> 40) & 0xffffu);
    const int i = (int)((k >> 8) & 15);
    const uint64_t S1 = samp[kk];
    if ((mask >> i) & 1u) {
      const uint64_t sidx = (d & ((1ull << 40) - 1)) + (uint64_t)__popc(mask & ((1u << i) - 1u));
      return S1 + v.ck32[v.cm->sparse[bv] + 256 * sidx + (k & 255)];
    }
    const uint32_t* sb = v.ck32 + v.cm->sub[bv] + 16 * kk;
    const uint64_t p0 = S1 + sb[i];
    if ((k & 255) == 0) return p0;
    // the sub-range ends at the next sub-sample, or at the range's end
    uint64_t p1 = (i + 1 < 16 && sb[i + 1] != 0xffffffffu) ? S1 + sb[i + 1] : 0;
    if (!p1) {
      const uint64_t ns = ((bv ? v.n - v.zeros : v.zeros) + 4095) / 4096;
      p1 = kk + 1 < ns ? samp[kk + 1] : v.n;
    }
    return dir_select<false>(v.bits, v.dir, bv, k, p0 >> 11, (p1 - 1) >> 11);
  }
  const uint64_t cnt = bv ? v.n - v.zeros : v.zeros;
  const uint64_t ns = (cnt + 4095) / 4096;
  const uint64_t idx = k >> 12;
  uint64_t lo = samp[idx] >> 11;
  uint64_t hi = (idx + 1 < ns) ? (samp[idx + 1] >> 11) : v.nsb - 1;
  auto before = [&](uint64_t s) -> uint64_t {
    const uint64_t z = v.dir[2 * s];
    return bv ? 2048 * s - z : z;
  };
  while (lo < hi) {
    const uint64_t mid = (lo + hi + 1) >> 1;
    if (before(mid) <= k) lo = mid;
    else hi = mid - 1;
  }
  return 2048 * lo + find_in_sb(v.bits, v.dir, lo, bv, (uint32_t)(k - before(lo)));
}


__device__ uint64_t q_wm(const QStruct& S, int op, uint32_t c, uint64_t x) {
  const int L = S.L;
  if (op == 0) {
    if (x >= S.n) return NONE;
    uint64_t pos = x, sym = 0;
    for (int l = 0; l < L; l++) {
      const BinLevel v = bin_level(S, l);
      const int b = get_bit(v, pos);
      sym = (sym << 1) | (uint64_t)b;
      pos = b ? v.zeros + rank1(v, pos) : rank0(v, pos);
    }
    return sym;
  }
  if (c >= S.sigma) return NONE;
  if (op == 1) {
    if (x >= S.n) return NONE;
    uint64_t s = 0, j = x + 1;
    for (int l = 0; l < L; l++) {
      const BinLevel v = bin_level(S, l);
      const int b = (c >> (L - 1 - l)) & 1;
      if (b) { s = v.zeros + rank1(v, s); j = v.zeros + rank1(v, j); }
      else { s = rank0(v, s); j = rank0(v, j); }
    }
    return j - s;
  }
  if (x == 0) return NONE;
  uint64_t s = 0, e = S.n;
  for (int l = 0; l < L; l++) {
    const BinLevel v = bin_level(S, l);
    const int b = (c >> (L - 1 - l)) & 1;
    if (b) { s = v.zeros + rank1(v, s); e = v.zeros + rank1(v, e); }
    else { s = rank0(v, s); e = rank0(v, e); }
  }
  if (x > e - s) return NONE;
  uint64_t pos = s + x - 1;
  for (int l = L - 1; l >= 0; l--) {
    const BinLevel v = bin_level(S, l);
    const int b = (c >> (L - 1 - l)) & 1;
    pos = b ? select_b(v, 1, pos - v.zeros) : select_b(v, 0, pos);
  }
  return pos;
}

__device__ uint64_t q_wt(const QStruct& S, int op, uint32_t c, uint64_t x) {
  const int L = S.L;
  if (op == 0) {
    if (x >= S.n) return NONE;
    uint64_t s = 0, e = S.n, pos = x, sym = 0;
    for (int l = 0; l < L; l++) {
      const BinLevel v = bin_level(S, l);
      const uint64_t zs = rank0(v, s), zp = rank0(v, pos), ze = rank0(v, e);
      const int b = get_bit(v, pos);
      sym = (sym << 1) | (uint64_t)b;
      if (!b) { pos = s + (zp - zs); e = s + (ze - zs); }
      else { pos = s + (ze - zs) + (pos - s) - (zp - zs); s = s + (ze - zs); }
    }
    return sym;
  }
  if (c >= S.sigma) return NONE;
  if (op == 1) {
    if (x >= S.n) return NONE;
    uint64_t s = 0, e = S.n, j = x + 1;
    for (int l = 0; l < L; l++) {
      const BinLevel v = bin_level(S, l);
      const uint64_t zs = rank0(v, s), zj = rank0(v, j), ze = rank0(v, e);
      const int b = (c >> (L - 1 - l)) & 1;
      if (!b) { j = s + (zj - zs); e = s + (ze - zs); }
      else { j = s + (ze - zs) + (j - s) - (zj - zs); s = s + (ze - zs); }
    }
    return j - s;
  }
  if (x == 0) return NONE;
  uint64_t S0[33];
  uint64_t s = 0, e = S.n;
  for (int l = 0; l < L; l++) {
    S0[l] = s;
    const BinLevel v = bin_level(S, l);
    const uint64_t zs = rank0(v, s), ze = rank0(v, e);
    const int b = (c >> (L - 1 - l)) & 1;
    if (!b) e = s + (ze - zs);
    else s = s + (ze - zs);
  }
  S0[L] = s;
  if (x > e - s) return NONE;
  uint64_t pos = s + x - 1;
  for (int l = L - 1; l >= 0; l--) {
    const BinLevel v = bin_level(S, l);
    const int b = (c >> (L - 1 - l)) & 1;
    const uint64_t off = pos - S0[l + 1];
    const uint64_t zs = rank0(v, S0[l]);
    pos = b ? select_b(v, 1, (S0[l] - zs) + off) : select_b(v, 0, zs + off);
  }
  return pos;
}

// Huffman-shaped tree: node (level l, prefix q) -> [start, end) on level l
__device__ __forceinline__ bool huff_node(const QStruct& S, int l, uint64_t q, uint64_t& st,
                                          uint64_t& en) {
  if (l >= S.L) return false;
  const uint64_t off = S.hq.node_lvl[3 * l], first = S.hq.node_lvl[3 * l + 1],
                 num = S.hq.node_lvl[3 * l + 2];
  if (q < first || q >= first + num) return false;
  st = S.hq.node[off + q - first];
  en = S.hq.node[off + q - first + 1];
  return true;
}

__device__ uint64_t q_huff(const QStruct& S, int op, uint32_t c, uint64_t x) {
  if (op == 0) {
    if (x >= S.n) return NONE;
    uint64_t q = 0, s = 0, pos = x;
    for (int l = 0; l < S.L; l++) {
      const BinLevel v = bin_level(S, l);
      const int b = get_bit(v, pos);
      const uint64_t child = (q << 1) | (uint64_t)b;
      const uint64_t cnt_b = b ? (pos - s) - (rank0(v, pos) - rank0(v, s)) : rank0(v, pos) - rank0(v, s);
      uint64_t cs, ce;
      if (!huff_node(S, l + 1, child, cs, ce)) {
        // a leaf at depth l+1: canonical code -> symbol
        const int ln = l + 1;
        const uint64_t first = S.hq.len_first[ln], base = S.hq.len_base[ln];
        return S.hq.sym_by_rank[base + (child - first)];
      }
      q = child;
      s = cs;
      pos = cs + cnt_b;
    }
    return NONE;
  }
  if (c >= S.sigma) return NONE;
  const int ln = S.hq.len[c];
  const uint64_t code = S.hq.code[c];
  if (op == 1) {
    if (x >= S.n) return NONE;
    if (ln == 0) return 0;
    uint64_t q = 0, s = 0, j = x + 1;
    for (int l = 0; l < ln; l++) {
      const BinLevel v = bin_level(S, l);
      const int b = (int)((code >> (ln - 1 - l)) & 1u);
      const uint64_t z = rank0(v, j) - rank0(v, s);
      const uint64_t cb = b ? (j - s) - z : z;
      if (l == ln - 1) return cb;
      q = (q << 1) | (uint64_t)b;
      uint64_t cs, ce;
      huff_node(S, l + 1, q, cs, ce);
      s = cs;
      j = cs + cb;
    }
    return NONE;
  }
  if (x == 0 || ln == 0) return NONE;
  uint64_t S0[33];
  uint64_t q = 0, s = 0, e = S.n;
  for (int l = 0; l < ln; l++) {
    S0[l] = s;
    const BinLevel v = bin_level(S, l);
    const int b = (int)((code >> (ln - 1 - l)) & 1u);
    const uint64_t z = rank0(v, e) - rank0(v, s);
    const uint64_t cb = b ? (e - s) - z : z;
    if (l == ln - 1) {
      if (x > cb) return NONE;
      break;
    }
    q = (q << 1) | (uint64_t)b;
    uint64_t cs, ce;
    huff_node(S, l + 1, q, cs, ce);
    s = cs;
    e = ce;
  }
  // bottom-up: at level l the target is the off-th b-bit of node [S0[l], .)
  uint64_t off = x - 1, pos = 0;
  for (int l = ln - 1; l >= 0; l--) {
    const BinLevel v = bin_level(S, l);
    const int b = (int)((code >> (ln - 1 - l)) & 1u);
    const uint64_t zs = rank0(v, S0[l]);
    pos = b ? select_b(v, 1, (S0[l] - zs) + off) : select_b(v, 0, zs + off);
    if (l > 0) off = pos - S0[l];
  }
  return pos;
}

// 4-ary tree: digit levels, per-value counts
struct DigLevel {
  const uint64_t* bits;
  const uint64_t* dir;
  const uint64_t* samp;  // 4 regions of n/4096 + 1: samples of values 0..3
  uint64_t n, nsb;
  const ClarkMeta* cm;
  const uint64_t* ck64;
  const uint32_t* ck32;
};

__device__ __forceinline__ DigLevel dig_level(const QStruct& S, int l) {
  const LevelMeta m = S.meta[l];
  DigLevel v;
  v.bits = S.bits + m.bit_off;
  v.dir = S.dir + m.dir_off;
  v.samp = S.samp + m.s0_off;
  v.n = m.n;
  v.nsb = m.nsb;
  v.cm = S.cmeta ? S.cmeta + l : nullptr;
  v.ck64 = S.ck64;
  v.ck32 = S.ck32;
  return v;
}

// count of digit d in [0, x)
__device__ uint64_t rank_d(const DigLevel& v, uint32_t d, uint64_t x) {
  const uint64_t s = x >> 10;
  const uint32_t b = (uint32_t)((x >> 8) & 3);
  uint64_t r = v.dir[8 * s + d] + ((v.dir[8 * s + 4 + b] >> (16 * d)) & 0xffffull);
  const uint64_t wend = x >> 5;
  for (uint64_t w = 32 * s + 8 * b; w < wend; w++) r += __popcll(digit_match(v.bits[w], d));
  const uint32_t rem = (uint32_t)(x & 31);
  if (rem) r += __popcll(digit_match(v.bits[wend], d) & ((1ull << (2 * rem)) - 1ull));
  return r;
}

__device__ __forceinline__ uint32_t get_digit(const DigLevel& v, uint64_t i) {
  return (uint32_t)((v.bits[i >> 5] >> (2 * (i & 31))) & 3ull);
}

// position of the k-th (0-based) occurrence of digit d; k < its count
// (Section 5.2 generalized select: the structures of the binary case per
// digit value)
__device__ uint64_t select_d(const DigLevel& v, uint32_t d, uint64_t k) {
  const uint64_t* samp = v.samp + d * (v.n / 4096 + 1);
  const uint64_t kk = k >> 12;
  if (v.cm) {
    // constant-time directory: stored answer, or a sub-range shorter than
    // 2^16 digits to search
    const uint64_t dsc = v.ck64[v.cm->desc[d] + kk];
    if (dsc >> 63) return v.ck64[v.cm->huge[d] + (dsc & ((1ull << 63) - 1)) + (k & 4095)];
    const uint32_t mask = (uint32_t)((dsc >> 40) & 0xffffu);
    const int i = (int)((k >> 8) & 15);
    const uint64_t S1 = samp[kk];
    if ((mask >> i) & 1u) {
      const uint64_t sidx = (dsc & ((1ull << 40) - 1)) + (uint64_t)__popc(mask & ((1u << i) - 1u));
      return S1 + v.ck32[v.cm->sparse[d] + 256 * sidx + (k & 255)];
    }
    const uint32_t* sb = v.ck32 + v.cm->sub[d] + 16 * kk;
    const uint64_t p0 = S1 + sb[i];
    if ((k & 255) == 0) return p0;
    // the sub-range ends at the next sub-sample, or at the range's end
    uint64_t p1 = (i + 1 < 16 && sb[i + 1] != 0xffffffffu) ? S1 + sb[i + 1] : 0;
    if (!p1) {
      const uint64_t ns = (v.dir[8 * v.nsb + d] + 4095) / 4096;
      p1 = kk + 1 < ns ? samp[kk + 1] : v.n;
    }
    return dir_select<true>(v.bits, v.dir, (int)d, k, p0 >> 10, (p1 - 1) >> 10);
  }
  // sampled: the search starts between two samples
  const uint64_t ns = (v.dir[8 * v.nsb + d] + 4095) / 4096;
  const uint64_t lo = samp[kk] >> 10;
  const uint64_t hi = kk + 1 < ns ? samp[kk + 1] >> 10 : v.nsb - 1;
  return dir_select<true>(v.bits, v.dir, (int)d, k, lo, hi);
}

__device__ uint64_t q_multi(const QStruct& S, int op, uint32_t c, uint64_t x) {
  const int L = S.L, D = S.levels;
  auto dwidth = [&](int be) { return (2 * be + 1 < L) ? 2 : 1; };
  auto cdigit = [&](int be) -> uint32_t {
    const int w = dwidth(be);
    const int sh = L - 2 * be - w;
    return (c >> sh) & ((1u << w) - 1u);
  };
  if (op == 0) {
    if (x >= S.n) return NONE;
    uint64_t s = 0, e = S.n, pos = x, sym = 0;
    for (int be = 0; be < D; be++) {
      const DigLevel v = dig_level(S, be);
      const uint32_t d = get_digit(v, pos);
      sym = (sym << dwidth(be)) | d;
      uint64_t cs = s;
      for (uint32_t d2 = 0; d2 < d; d2++) cs += rank_d(v, d2, e) - rank_d(v, d2, s);
      const uint64_t rs = rank_d(v, d, s);
      const uint64_t ne = cs + (rank_d(v, d, e) - rs);
      pos = cs + (rank_d(v, d, pos) - rs);
      s = cs;
      e = ne;
    }
    return sym;
  }
  if (c >= S.sigma) return NONE;
  if (op == 1) {
    if (x >= S.n) return NONE;
    uint64_t s = 0, e = S.n, j = x + 1;
    for (int be = 0; be < D; be++) {
      const DigLevel v = dig_level(S, be);
      const uint32_t d = cdigit(be);
      uint64_t cs = s;
      for (uint32_t d2 = 0; d2 < d; d2++) cs += rank_d(v, d2, e) - rank_d(v, d2, s);
      const uint64_t rs = rank_d(v, d, s);
      const uint64_t ne = cs + (rank_d(v, d, e) - rs);
      j = cs + (rank_d(v, d, j) - rs);
      s = cs;
      e = ne;
    }
    return j - s;
  }
  if (x == 0) return NONE;
  uint64_t S0[17];
  uint64_t s = 0, e = S.n;
  for (int be = 0; be < D; be++) {
    S0[be] = s;
    const DigLevel v = dig_level(S, be);
    const uint32_t d = cdigit(be);
    uint64_t cs = s;
    for (uint32_t d2 = 0; d2 < d; d2++) cs += rank_d(v, d2, e) - rank_d(v, d2, s);
    const uint64_t ne = cs + (rank_d(v, d, e) - rank_d(v, d, s));
    s = cs;
    e = ne;
  }
  S0[D] = s;
  if (x > e - s) return NONE;
  uint64_t pos = s + x - 1;
  for (int be = D - 1; be >= 0; be--) {
    const DigLevel v = dig_level(S, be);
    const uint32_t d = cdigit(be);
    const uint64_t off = pos - S0[be + 1];
    pos = select_d(v, d, rank_d(v, d, S0[be]) + off);
  }
  return pos;
}

__device__ uint64_t q_rs(const QStruct& S, int op, uint32_t c, uint64_t x) {
  const BinLevel v = bin_level(S, 0);
  if (op == 0) return x < S.n ? (uint64_t)get_bit(v, x) : NONE;
  if (c > 1) return NONE;
  if (op == 1) {
    if (x >= S.n) return NONE;
    return c ? rank1(v, x + 1) : rank0(v, x + 1);
  }
  const uint64_t cnt = c ? S.n - v.zeros : v.zeros;
  if (x == 0 || x > cnt) return NONE;
  return select_b(v, (int)c, x - 1);
}

__global__ void k_query(QStruct S, int op, const uint32_t* c, const uint64_t* x, uint64_t q,
                        uint64_t* out) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= q) return;
  const uint32_t ci = c ? c[i] : 0u;
  const uint64_t xi = x[i];
  uint64_t r;
  switch (S.kind) {
    case WT_KIND_WM: r = q_wm(S, op, ci, xi); break;
    case WT_KIND_WT: r = q_wt(S, op, ci, xi); break;
    case WT_KIND_HUFF: r = q_huff(S, op, ci, xi); break;
    case WT_KIND_MULTI: r = q_multi(S, op, ci, xi); break;
    default: r = q_rs(S, op, ci, xi); break;
  }
  out[i] = r;
}

static void fill_qstruct(const wt_struct* h, QStruct& S) {
  S.kind = h->kind;
  S.n = h->n;
  S.sigma = h->sigma;
  S.L = (int)h->L;
  S.levels = (int)h->levels;
  S.bits = h->d_bits_ro;
  S.dir = h->d_dir;
  S.samp = h->d_samp;
  S.meta = h->d_meta;
  S.zeros = h->d_zeros;
  S.hq.code = h->d_code;
  S.hq.len = h->d_len;
  S.hq.sym_by_rank = h->d_sym_by_rank;
  S.hq.len_first = h->d_len_tab;
  S.hq.len_base = h->d_len_tab ? h->d_len_tab + 34 : nullptr;
  S.hq.len_count = h->d_len_tab ? h->d_len_tab + 68 : nullptr;
  S.hq.node = h->d_node;
  S.hq.node_lvl = h->d_node_lvl;
  S.cmeta = h->d_cmeta;
  S.ck64 = h->d_ck64;
  S.ck32 = h->d_ck32;
}

wt_status launch_query(wt_struct* h, int op, const uint32_t* c, const uint64_t* x, uint64_t q,
                       uint64_t* out, cudaStream_t st) {
  if (q == 0) return WT_OK;
  QStruct S;
  fill_qstruct(h, S);
  k_query<<<(unsigned)((q + 127) / 128), 128, 0, st>>>(S, op, c, x, q, out);
  count_launch();
  CK(cudaGetLastError());
  return WT_OK;
}

// Queries over several structures in one launch: query i applies op[i] to
// structure sid[i] of the table.
__global__ void k_query_multi(const QStruct* tab, uint32_t ns, const uint32_t* sid,
                              const uint8_t* op, const uint32_t* c, const uint64_t* x, uint64_t q,
                              uint64_t* out) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= q) return;
  const uint32_t s = sid[i];
  const int o = op[i];
  if (s >= ns || o > 2) {
    out[i] = NONE;
    return;
  }
  const QStruct& S = tab[s];
  const uint32_t ci = c[i];
  const uint64_t xi = x[i];
  uint64_t r;
  switch (S.kind) {
    case WT_KIND_WM: r = q_wm(S, o, ci, xi); break;
    case WT_KIND_WT: r = q_wt(S, o, ci, xi); break;
    case WT_KIND_HUFF: r = q_huff(S, o, ci, xi); break;
    case WT_KIND_MULTI: r = q_multi(S, o, ci, xi); break;
    default: r = q_rs(S, o, ci, xi); break;
  }
  out[i] = r;
}

wt_status launch_query_multi(wt_struct* const* hs, uint32_t nh, const uint32_t* sid,
                             const uint8_t* op, const uint32_t* c, const uint64_t* x, uint64_t q,
                             uint64_t* out, cudaStream_t st) {
  if (q == 0) return WT_OK;
  std::vector<QStruct> tab(std::max<uint32_t>(nh, 1));
  for (uint32_t i = 0; i < nh; i++) fill_qstruct(hs[i], tab[i]);
  Work wk{st, {}};
  QStruct* d_tab = nullptr;
  TRY(wk.get(&d_tab, tab.size()));
  TRY(upload(d_tab, tab.data(), tab.size() * sizeof(QStruct), st));
  k_query_multi<<<(unsigned)((q + 127) / 128), 128, 0, st>>>(d_tab, nh, sid, op, c, x, q, out);
  count_launch();
  CK(cudaGetLastError());
  return WT_OK;
}

}  // namespace wtk
