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

}  // namespace cfet
