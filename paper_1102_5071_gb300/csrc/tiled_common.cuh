// Window tiling of the matrix-free XXZ apply for chains whose vectors leave
// L2 (shared by the complex64 and fixed-point persistent kernels).
//
// The element-wise apply gathers 2N - 1 neighbours of every element; for
// vectors beyond the 129 MB L2 the far-bit gathers read DRAM.  The tiled form
// splits the bits of the index into windows and runs one pass per window over
// tiles of 2^B elements staged in shared memory (cp.async, double-buffered):
//   window 0 takes contiguous tiles (bits 0..B-1): diagonal, previous Krylov
//     vector, flips of bits 0..B-1, hops of bonds (i, i+1) for i <= B-2;
//   window w >= 1 takes strided tiles made of 2^c contiguous elements times
//     the 2^width values of its bits [b0, b0 + width), width <= 8,
//     b0 = B - 1 + 7 (w - 1), c = B - width: flips of bits b0+1 .. b0+width-1
//     and hops of bonds b0 .. b0+width-2, added to the partial result of the
//     earlier windows.
// Consecutive windows share one bit, so every bond lies inside one window.
// The kernels separate the windows by grid-wide exchanges.
#pragma once

#include <cuda_runtime.h>

namespace cfet {

constexpr int kHighWindow = 8;       // bits of a high window, its first shared with the window before
constexpr int kTiledMaxWindows = 4;  // chains of up to B + 3 * 7 sites

struct TileWin {
  int b0, width, c;
};

// Windows 1.. of an N-site chain with tiles of 2^TB elements; returns the
// number of windows including window 0 (W[0] unused).  This and tile_x also
// compile for the host, where cfet_selftest_tiling checks them.
template <int TB>
__host__ __device__ __forceinline__ int tiled_windows(int N, TileWin (&W)[kTiledMaxWindows]) {
  int n = 1;
  for (int b0 = TB - 1; b0 + 1 < N && n < kTiledMaxWindows; b0 += kHighWindow - 1, ++n) {
    const int width = (N - b0) < kHighWindow ? (N - b0) : kHighWindow;
    W[n].b0 = b0;
    W[n].width = width;
    W[n].c = TB - width;
  }
  return n;
}

// Element index of slot j of strided tile t of window W.
__host__ __device__ __forceinline__ int tile_x(const TileWin& W, int t, int j) {
  const int nb = W.b0 - W.c;  // bits [c, b0) come from t
  const int tl = t & ((1 << nb) - 1), th = t >> nb;
  return (j & ((1 << W.c) - 1)) | (tl << W.c) | ((j >> W.c) << W.b0) | (th << (W.b0 + W.width));
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
// Barrier of the n worker threads only (named barrier 1).
__device__ __forceinline__ void workers_sync(int n) { asm volatile("bar.sync 1, %0;" ::"r"(n) : "memory"); }
// Hand-over between the workers and the control warp around a window exchange
// (named barriers 2 and 3 over all threads of the CTA).
__device__ __forceinline__ void window_written_sync() { asm volatile("bar.sync 2;" ::: "memory"); }
__device__ __forceinline__ void window_exchanged_sync() { asm volatile("bar.sync 3;" ::: "memory"); }

// ------------------------------------------------------------------ TMA tile transfers
// Tensor maps of the tiled apply (built on the host over the whole Krylov
// basis; its vectors are contiguous, so the vector index continues the
// outermost dimension; every coordinate non-negative, the innermost 0).  For
// complex64 (one 8-byte word per element, tiles of 2^12):
//   window 0: (256, 2^(N-8) nvec) words, box (256, 16): tile t of vector v at
//     (0, 16 t + 2^(N-8) v) = elements [4096 t, 4096 t + 4096);
//   window w >= 1, c <= 8: (2^c, 2^(b0-c), 2^width, 2^(N-b0-width) nvec), box
//     (2^c, 1, 2^width, 1) at (0, tl, 0, th + 2^(N-b0-width) v), tile
//     t = (th << (b0 - c)) | tl;  c > 8: the low bits as (256, 2^(c-8)), box
//     (256, 2^(c-8), 1, 2^width, 1) at (0, 0, tl, 0, th + ...).
// The fixed-point maps count two words per element (tiles of 2^11): rows of
// 128 elements in window 0, the low dimension 2^(c+1) words (split at c > 7).
//   Shared memory holds the box with dimension 0 fastest: slot
//   (j & (2^c - 1)) | (window bits << c), the slot order of tile_x.
constexpr int kTmaMapBytes = 128;    // sizeof(CUtensorMap)
constexpr int kTmaStages = 3;        // tiles in flight per CTA

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// Make mbarrier.init visible to the other threads and to the async proxy (then a CTA barrier).
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Order this thread's generic-proxy accesses with later async-proxy (TMA) ones.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_all() { asm volatile("fence.proxy.async;" ::: "memory"); }
__device__ __forceinline__ void tma_load_2d(void* dst, const void* map, int c0, int c1, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"(map), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_4d(void* dst, const void* map, int c0, int c1, int c2, int c3,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
      ::"r"(smem_u32(dst)), "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_5d(void* dst, const void* map, int c0, int c1, int c2, int c3, int c4,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], [%7];"
      ::"r"(smem_u32(dst)), "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_store_2d(const void* map, int c0, int c1, const void* src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];"
               ::"l"(map), "r"(c0), "r"(c1), "r"(smem_u32(src))
               : "memory");
}
__device__ __forceinline__ void tma_store_4d(const void* map, int c0, int c1, int c2, int c3, const void* src) {
  asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4}], [%5];"
               ::"l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(src))
               : "memory");
}
__device__ __forceinline__ void tma_store_5d(const void* map, int c0, int c1, int c2, int c3, int c4,
                                             const void* src) {
  asm volatile("cp.async.bulk.tensor.5d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4, %5}], [%6];"
               ::"l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(src))
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Wait until at most one committed store group still reads shared memory.
__device__ __forceinline__ void bulk_wait_read_1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
// Wait until every committed store group has completed its writes.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Tile t of window W (first: window 0) of vector v of an N-site chain, tiles of
// 2^TB elements of WPE 8-byte words (1: complex64, 2: an int64 pair): TMA load
// into dst (bar completes with the bytes) and TMA store from src.  The maps view
// the basis in 8-byte words: window 0 as rows of 256 words (2^RS elements,
// RS = 8 - log2 WPE), a tile being 2^(TB - RS) rows; window w >= 1 as the
// tile's 2^c low elements (one box dimension while 2^c WPE <= 256 words, else
// 256 x 2^c WPE / 256), bits [c, b0), the window's bits and the rest.
template <int TB, int WPE>
__device__ __forceinline__ void tile_load_t(void* dst, const void* map, bool first, const TileWin& W, int N, int t,
                                            int v, unsigned long long* bar) {
  constexpr int RS = WPE == 2 ? 7 : 8;
  if (first) {
    tma_load_2d(dst, map, 0, (t << (TB - RS)) + v * (1 << (N - RS)), bar);
    return;
  }
  const int nb = W.b0 - W.c, tl = t & ((1 << nb) - 1), th = (t >> nb) + v * (1 << (N - W.b0 - W.width));
  if (W.c <= RS) tma_load_4d(dst, map, 0, tl, 0, th, bar);
  else tma_load_5d(dst, map, 0, 0, tl, 0, th, bar);
}
template <int TB, int WPE>
__device__ __forceinline__ void tile_store_t(const void* map, bool first, const TileWin& W, int N, int t, int v,
                                             const void* src) {
  constexpr int RS = WPE == 2 ? 7 : 8;
  if (first) {
    tma_store_2d(map, 0, (t << (TB - RS)) + v * (1 << (N - RS)), src);
    return;
  }
  const int nb = W.b0 - W.c, tl = t & ((1 << nb) - 1), th = (t >> nb) + v * (1 << (N - W.b0 - W.width));
  if (W.c <= RS) tma_store_4d(map, 0, tl, 0, th, src);
  else tma_store_5d(map, 0, 0, tl, 0, th, src);
}
// The complex64 kernel's tiles: 2^12 elements of one word.
__device__ __forceinline__ void tile_load(void* dst, const void* map, bool first, const TileWin& W, int N, int t,
                                          int v, unsigned long long* bar) {
  tile_load_t<12, 1>(dst, map, first, W, N, t, v, bar);
}
__device__ __forceinline__ void tile_store(const void* map, bool first, const TileWin& W, int N, int t, int v,
                                           const void* src) {
  tile_store_t<12, 1>(map, first, W, N, t, v, src);
}

}  // namespace cfet
