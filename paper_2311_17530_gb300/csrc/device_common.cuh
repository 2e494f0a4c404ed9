// Device helpers shared by the fill and traceback kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace msadp {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int ld_acquire(const int32_t *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed(const int32_t *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(int32_t *p, int v) {
    asm volatile("st.relaxed.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void st_release(int32_t *p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ int ld_volatile(const int32_t *p) {
    return *reinterpret_cast<const volatile int32_t *>(p);
}

// Bounded wait until *flag >= need. Returns false when the launch status is set
// by another warp or when the wait exceeds spin_ns (then the caller records
// MSA_ETIMEOUT and leaves). Never traps; every exit path is finite.
__device__ __forceinline__ bool wait_at_least(const int32_t *flag, int need, const int32_t *err,
                                              int64_t spin_ns) {
    if (ld_acquire(flag) >= need) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1; it < (1u << 27); ++it) {
        if (ld_acquire(flag) >= need) return true;
        if ((it & 31) == 0) {
            if (ld_volatile(err) != 0) return false;
            if ((int64_t)(global_ns() - t0) > spin_ns) return false;
        }
        __nanosleep(it < 64 ? 32 : 256);
    }
    return false;
}

// Geometry of the generic tile kernel (compile-time per k and tile edge E).
//
// The halo'd score tile in shared memory is laid out with strides
// sh_{K-1} = 1, sh_j = sh_{j+1} (ext_{j+1} + 1) + pad_j: a predecessor is still a
// constant offset away, and the pads (found by counting, for each shape, the
// shared-memory wavefronts of the predecessor reads of every round of 32 cells)
// spread the cells of a plane over more of the 32 banks than power-of-two
// strides do. Positions inside the pads are never read or written.
__host__ __device__ constexpr int geo_pad(int K, int E, int j) {
    constexpr int none = 0;
    return K == 4 && E == 5   ? (j == 1 ? 1 : none)
         : K == 4 && E == 6   ? (j == 0 ? 5 : j == 1 ? 5 : none)
         : K == 5 && E == 3   ? (j == 1 ? 3 : none)
         : K == 5 && E == 4   ? (j == 0 ? 1 : j == 1 ? 1 : j == 2 ? 3 : none)
         : K == 6 && E == 2   ? (j == 1 ? 1 : j == 2 ? 1 : none)
         : K == 6 && E == 3   ? (j == 1 ? 3 : none)
         : K == 3 && E == 12  ? (j == 0 ? 1 : j == 1 ? 1 : none)
                              : none;
}
// halo'd tile stride of axis i; i = -1 gives the tile's size sh_0 (ext_0 + 1)
__host__ __device__ constexpr int geo_sh(int K, int E, int i) {
    int s = 1;
    for (int j = K - 2; j >= i; --j) s = s * (tile_ext(K, E, j + 1) + 1) + (j >= 0 ? geo_pad(K, E, j) : 0);
    return s;
}
__host__ __device__ constexpr int geo_cellsh(int K, int E) {  // cells of the halo'd tile
    int s = 1;
    for (int j = 0; j < K; ++j) s *= tile_ext(K, E, j) + 1;
    return s;
}
__host__ __device__ constexpr int geo_st(int K, int E, int i) {  // interior tile stride
    int s = 1;
    for (int j = K - 1; j > i; --j) s *= tile_ext(K, E, j);
    return s;
}
__host__ __device__ constexpr int geo_volh(int K, int E) { return geo_sh(K, E, -1); }
__host__ __device__ constexpr int geo_vol(int K, int E) { return geo_st(K, E, -1); }
__host__ __device__ constexpr int geo_planes(int K, int E) {
    int s = 0;
    for (int i = 0; i < K; ++i) s += tile_ext(K, E, i);
    return s - K + 1;
}
__host__ __device__ constexpr int geo_codes(int K, int E) {
    int s = 0;
    for (int i = 0; i < K; ++i) s += tile_ext(K, E, i);
    return s;
}
__host__ __device__ constexpr int geo_code_base(int K, int E, int i) {
    int s = 0;
    for (int j = 0; j < i; ++j) s += tile_ext(K, E, j);
    return s;
}
// smem offset of the predecessor x - e_m relative to x
__host__ __device__ constexpr int move_soff(int K, int E, int m) {
    int s = 0;
    for (int i = 0; i < K; ++i)
        if ((m >> i) & 1) s += geo_sh(K, E, i);
    return s;
}
// cells of halo face f: first axis at local -1 is f
__host__ __device__ constexpr int face_extent(int K, int E, int f, int j) {
    return j < f ? tile_ext(K, E, j) : (j == f ? 1 : tile_ext(K, E, j) + 1);
}
__host__ __device__ constexpr int face_size(int K, int E, int f) {
    int s = 1;
    for (int j = 0; j < K; ++j) s *= face_extent(K, E, f, j);
    return s;
}
__host__ __device__ constexpr int face_stride(int K, int E, int f, int i) {
    int s = 1;
    for (int j = K - 1; j > i; --j) s *= face_extent(K, E, f, j);
    return s;
}
__host__ __device__ constexpr int popc_c(int m) {
    int c = 0;
    while (m) {
        c += m & 1;
        m >>= 1;
    }
    return c;
}
__host__ __device__ constexpr int highbit_c(int m) {
    int h = -1;
    while (m) {
        m >>= 1;
        ++h;
    }
    return h;
}
__host__ __device__ constexpr int lowbit_c(int m) {  // index of the lowest set bit
    int l = 0;
    while (m && !(m & 1)) {
        m >>= 1;
        ++l;
    }
    return l;
}
__host__ __device__ constexpr int round_up(int x, int a) { return (x + a - 1) / a * a; }

}  // namespace msadp
