// wt_internal.cuh -- device-side types and helpers shared by the kernels of
// the GB300 wavelet library (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace wtk {

constexpr int TAU_MAX = 8;                  // levels per partition pass (upper bound)
constexpr int NCLS = 1 << (TAU_MAX + 1);    // class-tree slots: level j class k at 2^j-1+k
constexpr uint32_t FULL = 0xffffffffu;

// device error word bits
// (ERR_INTERNAL: a prefix table disagreed with a tile; never for correct tables)
// (ERR_STALL: a staged tile load did not complete within its time limit)
enum : uint32_t { ERR_SYMBOL = 1u, ERR_INTERNAL = 4u, ERR_STALL = 8u };

// structure shapes handled by the partition pass
enum Shape : int { SHAPE_WM = 0, SHAPE_WT = 1, SHAPE_HUFF = 2 };

// One tile of a pass: `count` consecutive elements of T_a starting at
// `start`, all inside node `node` (bit 31 of `flags`: first tile of its node).
struct TileDesc {
  uint64_t start;
  uint32_t count;
  uint32_t node;
  uint32_t first;
  uint32_t seg0;  // index of the node's first tile
};

// Per-tile digit counts of a pass (the K sub-problems' per-node counts of
// Section 4.2) and their prefix sums across tiles: tile ti's counts sit at
// tcnt[ti * tcs + r] (u32, exclusive within its chunk of TCHUNK tiles
// after the scan) and the chunk's exclusive counts at tchunk[c * tcs + r]
// (u64).
constexpr int TC_STRIDE = 256;  // the largest stride (t = 8)
// the stride of a pass's tables: its digit values, at least one warp's worth
__host__ __device__ inline uint32_t tc_stride(int t) { return t >= 5 ? (1u << t) : 32u; }
constexpr uint32_t TCHUNK = 256;

// Symbols per tile of the partition pass.
#ifndef WT_PASS_T
#define WT_PASS_T 4096
#endif
constexpr int PASS_T = WT_PASS_T;

// Batched builds: the per-sequence part of a pass, one entry per sequence
// taking part in the launch.  Its tiles are tile0 .. tile0 + ceil(n/T) - 1 of
// the launch's tile numbering.
// The pass's class starts (wm_cls) and the sequence's zero counts (zeros) are
// planned on the device from the totals of the pass's own tile counts;
// sigma (first pass only, else 0) is the bound the tile counts check the
// symbols against.
struct SegDesc {
  const void* in;
  void* out;
  uint64_t* bits;
  const uint64_t* lvl_off;
  const uint64_t* lvl_len;
  uint64_t* wm_cls;
  uint64_t* zeros;
  uint32_t* err;
  uint64_t n;
  uint32_t tile0;
  uint32_t sigma;
  int in_w, out_w, L, a, t, rbits;
};

struct PassParams {
  // input sequence T_a (elements hold the rbits = L - a low bits still needed)
  const void* in;
  int in_w;                 // bytes per input element (1, 2, 4)
  const uint32_t* code_map; // HUFF first pass: symbol -> left-aligned codeword
  // output sequence T_{a+t}, narrowed to rbits - t bits (nullptr on the last pass)
  void* out;
  int out_w;
  // geometry
  int L;                    // total levels (max code length for HUFF)
  int a, t;                 // first level of the pass, levels in the pass
  int rbits;                // bits per input element that matter (L - a)
  int shape;
  int digits;               // 1: emit 2-bit digit levels at even levels (multiary)
  // outputs
  uint64_t* bits;           // level bitmaps (or digit levels)
  const uint64_t* lvl_off;  // word offset per output level
  const uint64_t* lvl_len;  // elements per output level
  // class starts
  const uint64_t* wm_cls;   // WM: per level j of the pass, 2^j+1 starts at 2^j-1+j
  const uint64_t* wt_C;     // WT: C[v] = #symbols < v, v in [0, 2^L]
  const uint64_t* hf_node;  // HUFF: starts of the internal nodes, per level + sentinel
  const uint64_t* hf_lvl;   // HUFF: per level l: [3l] table offset, [3l+1] first internal prefix, [3l+2] count
  // tiles
  const TileDesc* tiles;    // nullptr: uniform tiles of TILE elements over n_in
  const uint32_t* ntiles_dev;
  uint32_t ntiles;
  uint64_t n_in;
  uint32_t tile0;           // first tile of the sequence (0 unless batched)
  uint32_t sigma;           // batched first passes: the tile counts check S[i] < sigma
  // batched builds: per-sequence parts, sorted by tile0
  const SegDesc* segs;
  uint32_t nsegs;
  // prefix sums of the tiles' digit counts (see TileDesc)
  const uint32_t* tcnt;
  const uint64_t* tchunk;
  uint32_t tcs;          // their stride (tc_stride of the largest digit width)
  uint32_t* ticket;      // tiles are taken in order from this counter
  uint32_t* err;
  // 16-byte units of a later pass's levels to zero, `clear_per` of them per
  // tile (nullptr: none); see clear_share
  uint4* clear;
  uint64_t clear_units, clear_per;
};

// Zero tile ti's share of `units` 16-byte units at `p`: units
// [ti * per, (ti + 1) * per), per = ceil(units / tiles) taken on the host.
__device__ __forceinline__ void clear_share(uint4* p, uint64_t units, uint64_t per, uint64_t ti,
                                            int tid, int nthreads) {
  const uint64_t b = ti * per;
  const uint64_t e = b + per < units ? b + per : units;
  for (uint64_t i = b + (uint64_t)tid; i < e; i += (uint64_t)nthreads)
    __stcs(p + i, make_uint4(0u, 0u, 0u, 0u));
}

__device__ __forceinline__ uint32_t rev_bits(uint32_t k, int j) {
  return j == 0 ? 0u : (__brev(k) >> (32 - j));
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// ---- bulk copies (TMA) into shared memory, completed on an mbarrier -------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// an mbarrier for one arriving thread, visible to the bulk-copy unit
__device__ __forceinline__ void mbar_init1(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Copy `bytes` (a multiple of 16; both addresses 16-byte aligned) from global
// memory to shared memory with the bulk-copy unit; the barrier's current
// phase completes when the bytes have landed.  One thread issues it.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// order this thread's earlier shared-memory accesses before later bulk copies
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for the phase of `bar` with parity `parity` to complete: false if it
// has not after about one second (or 2^24 polls), which a bulk copy of a few
// KB from valid memory never takes.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_addr(bar);
  uint64_t t0 = 0;
  for (uint32_t it = 0; it < (1u << 24); it++) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    if (it == 0) t0 = global_ns();
    else if (global_ns() - t0 > 1000000000ull) return false;
  }
  return false;
}


}  // namespace wtk
