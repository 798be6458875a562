// Building blocks shared by the stencil kernels: tile geometry of the 2.5D
// blocking and 16-byte vector loads and stores.
#pragma once

#include <cuda_runtime.h>

namespace rtm {

template <int R>
struct Tile {
    static constexpr int BX = 16;          // threads along x, 4 floats each
    static constexpr int BY = 16;          // threads along y
    static constexpr int TX = 4 * BX;      // 64 floats
    static constexpr int TY = BY;          // 16 rows
    static constexpr int SW = TX + 2 * R;  // shared row width (floats)
    static constexpr int SH = TY + 2 * R;  // shared rows
    static constexpr int HX = R / 4;       // halo vectors per side per row
    static_assert(R % 4 == 0, "radius must be a multiple of 4");
    static_assert(TY >= 2 * R, "tile too short for the y halo assignment");
};

struct F4 {
    float v[4];
};

__device__ __forceinline__ F4 zero4() { return F4{{0.f, 0.f, 0.f, 0.f}}; }

// cache-coherent at L2 (for data other blocks of the same launch write)
__device__ __forceinline__ F4 ld_l2(const float* p) {
    float4 t = __ldcg(reinterpret_cast<const float4*>(p));
    return F4{{t.x, t.y, t.z, t.w}};
}
__device__ __forceinline__ F4 ld_keep(const float* p) {  // read-only, keep in cache
    float4 t = __ldg(reinterpret_cast<const float4*>(p));
    return F4{{t.x, t.y, t.z, t.w}};
}
__device__ __forceinline__ F4 ld_stream(const float* p) {  // read once
    float4 t = __ldcs(reinterpret_cast<const float4*>(p));
    return F4{{t.x, t.y, t.z, t.w}};
}
__device__ __forceinline__ void st_stream(float* p, const F4& v) {
    __stcs(reinterpret_cast<float4*>(p), make_float4(v.v[0], v.v[1], v.v[2], v.v[3]));
}
__device__ __forceinline__ void st_plain4(float* p, const F4& v) {
    *reinterpret_cast<float4*>(p) = make_float4(v.v[0], v.v[1], v.v[2], v.v[3]);
}
__device__ __forceinline__ F4 lds4(const float* p) {
    float4 t = *reinterpret_cast<const float4*>(p);
    return F4{{t.x, t.y, t.z, t.w}};
}
__device__ __forceinline__ void sts4(float* p, const F4& v) {
    *reinterpret_cast<float4*>(p) = make_float4(v.v[0], v.v[1], v.v[2], v.v[3]);
}

}  // namespace rtm
