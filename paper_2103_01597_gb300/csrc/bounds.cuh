// Optional bounds checking of global indices (build with -DAC_BOUNDS_CHECK; off
// in the library's normal build, where the macros below cost nothing).  Every
// global index the stencil, substep and convolution kernels form is compared
// with its array's extent; an index outside it is recorded in a device word of
// the translation unit (the first one wins: tag and index) and the access is
// redirected to element 0 of the same array or skipped, so that the checked
// build itself stays in bounds.  The host reads and clears the words with
// ac_bounds_check_take().
#pragma once

#include <cuda_runtime.h>

#ifdef AC_BOUNDS_CHECK
namespace ac {
static __device__ unsigned long long bc_word;

// [i, i + count) inside [0, lim)?  Records the first violation.
__device__ __forceinline__ bool bc_ok(long long i, long long count, long long lim, unsigned tag) {
    if (i >= 0 && i + count <= lim) return true;
    atomicCAS(&bc_word, 0ull,
              (1ull << 63) | ((unsigned long long)(tag & 0x7fffu) << 48) |
                  ((unsigned long long)i & 0xffffffffffffull));
    return false;
}

// Read and clear this translation unit's word (host).
static inline unsigned long long bc_take_local() {
    unsigned long long w = 0, z = 0;
    if (cudaMemcpyFromSymbol(&w, bc_word, sizeof w) != cudaSuccess) return ~0ull;
    cudaMemcpyToSymbol(bc_word, &z, sizeof z);
    return w;
}
}  // namespace ac
// One reader per translation unit (its word is file-local): AC_BC_READER(name)
// defines ac::name() returning and clearing it.
#define AC_BC_READER(name) \
    namespace ac {         \
    unsigned long long name() { return bc_take_local(); } \
    }
#define AC_BC(i, lim, tag) (::ac::bc_ok((long long)(i), 1, (long long)(lim), (tag)) ? (i) : 0)
#define AC_BC_RANGE(i, count, lim, tag) ::ac::bc_ok((long long)(i), (count), (long long)(lim), (tag))
#define AC_BC_ONLY(...) __VA_ARGS__
#else
#define AC_BC(i, lim, tag) (i)
#define AC_BC_RANGE(i, count, lim, tag) true
#define AC_BC_ONLY(...)
#define AC_BC_READER(name)
#endif

// Tags of the checked index kinds (the bits 48..62 of a recorded word).
enum {
    AC_BC_STENCIL = 1,   // a stencil point or the cell itself (IdxPeriodicR, IdxPadded)
    AC_BC_TILE_IN = 2,   // a staged row of the binary32 tiled kernel
    AC_BC_TILE_W = 3,    // an accumulator element of the tiled kernel
    AC_BC_TILE_OUT = 4,  // an output element of the tiled kernel
    AC_BC_CONV_ACT = 5,  // a row-planar activation written by a convolution epilogue
    AC_BC_CONV_OUT = 6,  // a channel-major output of the last convolution
};
