// Snapshot-compression autoencoder on the tensor cores.
//
// Network (activations channels-last [z][y][x][c], bfloat16 between layers,
// float32 accumulation):
//   x0 = s / rms(s)
//   E1 patch conv 1->32 (kernel 2, stride 2) + LeakyReLU(0.1)   h1  [n/2]^3 x 32
//   E2 conv 32->16 (kernel 3, stride 2, padding 1)              lat [n/4]^3 x 16
//   D1 transposed conv 16->32 (kernel 4, stride 2, padding 1)
//      + LeakyReLU(0.1)                                          g1  [n/2]^3 x 32
//   D2 transposed patch conv 32->1 (kernel 2, stride 2)          y   [n]^3
//   s_hat = rms(s) * y
// A float32 snapshot becomes 16 bfloat16 channels per 4^3 voxels: 8x fewer
// bytes. Every convolution (forward, data gradient, weight gradient) is an
// implicit GEMM on the tcgen05 engine of tc_gemm.cuh; the rank-8 patch-conv
// weight gradients, bias gradients, loss and Adam run on the CUDA cores.
//
// Parameters: one float32 vector, in order W1[32][2][2][2], b1[32],
// W2[16][3][3][3][32], b2[16], W3[32][4][4][4][16], b3[32], W4[2][2][2][32],
// b4[1]; weights are rounded to bfloat16 when they are staged for the MMA.

#include <cuda_bf16.h>
#include <math.h>

#include "ae_internal.h"
#include "tc_gemm.cuh"

namespace rtm {
namespace ae {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ float leaky(float a) { return a > 0.f ? a : kSlope * a; }

__device__ __forceinline__ void decode3(long long v, int nx, int ny, int& x, int& y, int& z) {
    x = (int)(v % nx);
    const long long t = v / nx;
    y = (int)(t % ny);
    z = (int)(t / ny);
}

__device__ __forceinline__ uint4 zero4u() { return make_uint4(0, 0, 0, 0); }

__device__ __forceinline__ void bf16x8_to_f(const uint4& u, float* f) {
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
    for (int i = 0; i < 4; i++) {
        float2 t = __bfloat1622float2(h[i]);
        f[2 * i] = t.x;
        f[2 * i + 1] = t.y;
    }
}

__device__ __forceinline__ void store_bf16_row(bf16* dst, const float* f, int n) {
    for (int j = 0; j < n; j += 8)
        *reinterpret_cast<uint4*>(dst + j) = tc::pack8(f + j);
}

// transposed conv (kernel 4, stride 2, padding 1): parity q, tap index tau
// -> input offset t and kernel index k: q=0: (0,1), (-1,3); q=1: (1,0), (0,2)
__device__ __forceinline__ void convt_tap(int q, int tau, int& t, int& k) {
    if (q == 0) {
        t = tau ? -1 : 0;
        k = tau ? 3 : 1;
    } else {
        t = tau ? 0 : 1;
        k = tau ? 2 : 0;
    }
}

// ============================================================================
// engine self-check: C[M][N] = A[M][K] * B[N][K]^T
// ============================================================================
template <int NN>
struct OpGemm {
    using Args = GemmArgs;
    static constexpr int N = NN;
    __device__ static void tile(const Args& a, int& m0, int& c0, int& c1) {
        m0 = blockIdx.x * 128;
        c0 = 0;
        c1 = a.K / 32;
    }
    __device__ static void load(const Args& a, int m0, int ch, uint8_t* sA, uint8_t* sB, int tid) {
        const int r = m0 + tid;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            uint4 v = zero4u();
            if (r < a.M)
                v = *reinterpret_cast<const uint4*>(a.A + (size_t)r * a.K + ch * 32 + j * 8);
            tc::st_vec8(sA, tid, j * 8, v);
        }
        if (tid < N * 4) {
            const int n = tid >> 2, j = tid & 3;
            uint4 v = *reinterpret_cast<const uint4*>(a.B + (size_t)n * a.K + ch * 32 + j * 8);
            tc::st_vec8(sB, n, j * 8, v);
        }
    }
    __device__ static void load_async(const Args& a, int m0, int ch, uint8_t* sA, uint8_t* sB,
                                      int tid) {
        const int r = m0 + tid;
        const bf16* src = r < a.M ? a.A + (size_t)r * a.K + ch * 32 : a.A;
#pragma unroll
        for (int j = 0; j < 4; j++) tc::cp_async16(sA, tid, j * 8, src + j * 8, r < a.M);
        if (tid < N * 4) {
            const int n = tid >> 2, j = tid & 3;
            uint4 v = *reinterpret_cast<const uint4*>(a.B + (size_t)n * a.K + ch * 32 + j * 8);
            tc::st_vec8(sB, n, j * 8, v);
        }
    }
    __device__ static void epilogue(const Args& a, int m0, int row, const float* acc) {
        const int r = m0 + row;
        if (r >= a.M) return;
        for (int n = 0; n < N; n++) a.C[(size_t)r * N + n] = acc[n];
    }
};

// ============================================================================
// forward layers
// ============================================================================
struct OpE1 {  // x0 (strided float32, scaled by 1/rms) -> h1
    using Args = E1Args;
    static constexpr int N = 32;
    __device__ static void tile(const Args&, int& m0, int& c0, int& c1) {
        m0 = blockIdx.x * 128;
        c0 = 0;
        c1 = 1;
    }
    __device__ static void load(const Args& a, int m0, int, uint8_t* sA, uint8_t* sB, int tid) {
        const long long v = m0 + tid;
        const long long total = (long long)a.h.nx * a.h.ny * a.h.nz;
        float f[8];
#pragma unroll
        for (int d = 0; d < 8; d++) f[d] = 0.f;
        if (v < total) {
            int x, y, z;
            decode3(v, a.h.nx, a.h.ny, x, y, z);
            const float s = *a.inv_sigma;
#pragma unroll
            for (int d = 0; d < 8; d++) {
                const int dz = d >> 2, dy = (d >> 1) & 1, dx = d & 1;
                f[d] = a.in.p[(long long)(2 * z + dz) * a.in.sz + (long long)(2 * y + dy) * a.in.sy +
                              2 * x + dx] *
                       s;
            }
        }
        tc::st_vec8(sA, tid, 0, tc::pack8(f));
        tc::st_vec8(sA, tid, 8, zero4u());
        tc::st_vec8(sA, tid, 16, zero4u());
        tc::st_vec8(sA, tid, 24, zero4u());
        if (tid < 32) {
            float w[8];
#pragma unroll
            for (int d = 0; d < 8; d++) w[d] = a.P[kOW1 + tid * 8 + d];
            tc::st_vec8(sB, tid, 0, tc::pack8(w));
            tc::st_vec8(sB, tid, 8, zero4u());
            tc::st_vec8(sB, tid, 16, zero4u());
            tc::st_vec8(sB, tid, 24, zero4u());
        }
    }
    __device__ static void epilogue(const Args& a, int m0, int row, const float* acc) {
        const long long v = m0 + row;
        if (v >= (long long)a.h.nx * a.h.ny * a.h.nz) return;
        float f[32];
#pragma unroll
        for (int c = 0; c < 32; c++) f[c] = leaky(acc[c] + a.P[kOB1 + c]);
        store_bf16_row(a.h1 + v * 32, f, 32);
    }
};

struct OpE2 {  // h1 -> latent
    using Args = E2Args;
    static constexpr int N = 16;
    __device__ static void tile(const Args&, int& m0, int& c0, int& c1) {
        m0 = blockIdx.x * 128;
        c0 = 0;
        c1 = 27;
    }
    __device__ static void load(const Args& a, int m0, int tap, uint8_t* sA, uint8_t* sB, int tid) {
        const long long v = m0 + tid;
        const long long total = (long long)a.l.nx * a.l.ny * a.l.nz;
        const int kz = tap / 9, ky = (tap / 3) % 3, kx = tap % 3;
        uint4 r[4] = {zero4u(), zero4u(), zero4u(), zero4u()};
        if (v < total) {
            int x, y, z;
            decode3(v, a.l.nx, a.l.ny, x, y, z);
            const int sx = 2 * x + kx - 1, sy = 2 * y + ky - 1, sz = 2 * z + kz - 1;
            if (sx >= 0 && sx < a.h.nx && sy >= 0 && sy < a.h.ny && sz >= 0 && sz < a.h.nz) {
                const uint4* src = reinterpret_cast<const uint4*>(
                    a.h1 + (((long long)sz * a.h.ny + sy) * a.h.nx + sx) * 32);
#pragma unroll
                for (int j = 0; j < 4; j++) r[j] = src[j];
            }
        }
#pragma unroll
        for (int j = 0; j < 4; j++) tc::st_vec8(sA, tid, 8 * j, r[j]);
        load_b(a, tap, sB, tid);
    }
    __device__ static void load_b(const Args& a, int tap, uint8_t* sB, int tid) {
        if (tid < 64) {
            const int o = tid >> 2, j = tid & 3;
            float w[8];
#pragma unroll
            for (int e = 0; e < 8; e++) w[e] = a.P[kOW2 + o * 864 + tap * 32 + 8 * j + e];
            tc::st_vec8(sB, o, 8 * j, tc::pack8(w));
        }
    }
    __device__ static void load_async(const Args& a, int m0, int tap, uint8_t* sA, uint8_t* sB,
                                      int tid) {
        const long long v = m0 + tid;
        const long long total = (long long)a.l.nx * a.l.ny * a.l.nz;
        const int kz = tap / 9, ky = (tap / 3) % 3, kx = tap % 3;
        const bf16* src = a.h1;
        bool ok = false;
        if (v < total) {
            int x, y, z;
            decode3(v, a.l.nx, a.l.ny, x, y, z);
            const int sx = 2 * x + kx - 1, sy = 2 * y + ky - 1, sz = 2 * z + kz - 1;
            if (sx >= 0 && sx < a.h.nx && sy >= 0 && sy < a.h.ny && sz >= 0 && sz < a.h.nz) {
                ok = true;
                src = a.h1 + (((long long)sz * a.h.ny + sy) * a.h.nx + sx) * 32;
            }
        }
#pragma unroll
        for (int j = 0; j < 4; j++) tc::cp_async16(sA, tid, 8 * j, src + 8 * j, ok);
        load_b(a, tap, sB, tid);
    }
    __device__ static void epilogue(const Args& a, int m0, int row, const float* acc) {
        const long long v = m0 + row;
        if (v >= (long long)a.l.nx * a.l.ny * a.l.nz) return;
        float f[16];
#pragma unroll
        for (int o = 0; o < 16; o++) f[o] = acc[o] + a.P[kOB2 + o];
        store_bf16_row(a.lat + v * 16, f, 16);
    }
};

struct OpD1 {  // latent -> g1, one output parity class per blockIdx.y
    using Args = D1Args;
    static constexpr int N = 32;
    __device__ static void tile(const Args&, int& m0, int& c0, int& c1) {
        m0 = blockIdx.x * 128;
        c0 = 0;
        c1 = 4;
    }
    __device__ static void load(const Args& a, int m0, int ch, uint8_t* sA, uint8_t* sB, int tid) {
        const int q = blockIdx.y, qz = q >> 2, qy = (q >> 1) & 1, qx = q & 1;
        const long long v = m0 + tid;
        const long long total = (long long)a.l.nx * a.l.ny * a.l.nz;
        int x = 0, y = 0, z = 0;
        if (v < total) decode3(v, a.l.nx, a.l.ny, x, y, z);
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int tau = 2 * ch + h;
            int tz, kz, ty, ky, tx, kx;
            convt_tap(qz, tau >> 2, tz, kz);
            convt_tap(qy, (tau >> 1) & 1, ty, ky);
            convt_tap(qx, tau & 1, tx, kx);
            uint4 r0 = zero4u(), r1 = zero4u();
            const int sx = x + tx, sy = y + ty, sz = z + tz;
            if (v < total && sx >= 0 && sx < a.l.nx && sy >= 0 && sy < a.l.ny && sz >= 0 &&
                sz < a.l.nz) {
                const uint4* src = reinterpret_cast<const uint4*>(
                    a.lat + (((long long)sz * a.l.ny + sy) * a.l.nx + sx) * 16);
                r0 = src[0];
                r1 = src[1];
            }
            tc::st_vec8(sA, tid, 16 * h, r0);
            tc::st_vec8(sA, tid, 16 * h + 8, r1);
        }
        load_b(a, ch, sB, tid);
    }
    __device__ static void load_async(const Args& a, int m0, int ch, uint8_t* sA, uint8_t* sB,
                                      int tid) {
        const int q = blockIdx.y, qz = q >> 2, qy = (q >> 1) & 1, qx = q & 1;
        const long long v = m0 + tid;
        const long long total = (long long)a.l.nx * a.l.ny * a.l.nz;
        int x = 0, y = 0, z = 0;
        if (v < total) decode3(v, a.l.nx, a.l.ny, x, y, z);
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int tau = 2 * ch + h;
            int tz, kz, ty, ky, tx, kx;
            convt_tap(qz, tau >> 2, tz, kz);
            convt_tap(qy, (tau >> 1) & 1, ty, ky);
            convt_tap(qx, tau & 1, tx, kx);
            const int sx = x + tx, sy = y + ty, sz = z + tz;
            const bool ok = v < total && sx >= 0 && sx < a.l.nx && sy >= 0 && sy < a.l.ny &&
                            sz >= 0 && sz < a.l.nz;
            const bf16* src = ok ? a.lat + (((long long)sz * a.l.ny + sy) * a.l.nx + sx) * 16 : a.lat;
            tc::cp_async16(sA, tid, 16 * h, src, ok);
            tc::cp_async16(sA, tid, 16 * h + 8, src + 8, ok);
        }
        load_b(a, ch, sB, tid);
    }
    __device__ static void load_b(const Args& a, int ch, uint8_t* sB, int tid) {
        const int q = blockIdx.y, qz = q >> 2, qy = (q >> 1) & 1, qx = q & 1;
        {
            const int o = tid >> 2, j = tid & 3, h = j >> 1, i0 = (j & 1) * 8;
            const int tau = 2 * ch + h;
            int tz, kz, ty, ky, tx, kx;
            convt_tap(qz, tau >> 2, tz, kz);
            convt_tap(qy, (tau >> 1) & 1, ty, ky);
            convt_tap(qx, tau & 1, tx, kx);
            const int ktap = (kz * 4 + ky) * 4 + kx;
            float w[8];
#pragma unroll
            for (int e = 0; e < 8; e++) w[e] = a.P[kOW3 + o * 1024 + ktap * 16 + i0 + e];
            tc::st_vec8(sB, o, 8 * j, tc::pack8(w));
        }
    }
    __device__ static void epilogue(const Args& a, int m0, int row, const float* acc) {
        const long long v = m0 + row;
        if (v >= (long long)a.l.nx * a.l.ny * a.l.nz) return;
        const int q = blockIdx.y, qz = q >> 2, qy = (q >> 1) & 1, qx = q & 1;
        int x, y, z;
        decode3(v, a.l.nx, a.l.ny, x, y, z);
        const long long o = (((long long)(2 * z + qz) * a.h.ny + (2 * y + qy)) * a.h.nx + 2 * x + qx);
        float f[32];
#pragma unroll
        for (int c = 0; c < 32; c++) f[c] = leaky(acc[c] + a.P[kOB3 + c]);
        store_bf16_row(a.g1 + o * 32, f, 32);
    }
};

// D1 with D2 fused into its epilogue (inference): each accumulator row is a
// g1 voxel (32 channels, rounded to bfloat16 as in the unfused pair), D2 maps
// it to its 2 x 2 x 2 output block, so g1 never goes to memory
struct OpD12 {
    using Args = D12Args;
    static constexpr int N = 32;
    __device__ static void tile(const Args& a, int& m0, int& c0, int& c1) {
        OpD1::tile(a.d1, m0, c0, c1);
    }
    __device__ static void load(const Args& a, int m0, int ch, uint8_t* sA, uint8_t* sB, int tid) {
        OpD1::load(a.d1, m0, ch, sA, sB, tid);
    }
    __device__ static void load_async(const Args& a, int m0, int ch, uint8_t* sA, uint8_t* sB,
                                      int tid) {
        OpD1::load_async(a.d1, m0, ch, sA, sB, tid);
    }
    // W4 rounded to bfloat16, staged once per CTA
    static constexpr int kExtraSmem = 256 * 4;
    __device__ static void load_extra(const Args& a, uint8_t* extra, int tid) {
        float* w = reinterpret_cast<float*>(extra);
        for (int i = tid; i < 256; i += 128)
            w[i] = __bfloat162float(__float2bfloat16_rn(a.d1.P[kOW4 + i]));
    }
    __device__ static void epilogue_x(const Args& a, int m0, int row, const float* acc,
                                      const uint8_t* extra) {
        epilogue_w(a, m0, row, acc, reinterpret_cast<const float*>(extra));
    }
    __device__ static void epilogue(const Args& a, int m0, int row, const float* acc) {
        float w4[256];
        for (int i = 0; i < 256; i++)
            w4[i] = __bfloat162float(__float2bfloat16_rn(a.d1.P[kOW4 + i]));
        epilogue_w(a, m0, row, acc, w4);
    }
    __device__ static void epilogue_w(const Args& a, int m0, int row, const float* acc,
                                      const float* w4) {
        const D1Args& d = a.d1;
        const long long v = m0 + row;
        if (v >= (long long)d.l.nx * d.l.ny * d.l.nz) return;
        const int q = blockIdx.y, qz = q >> 2, qy = (q >> 1) & 1, qx = q & 1;
        int x, y, z;
        decode3(v, d.l.nx, d.l.ny, x, y, z);
        const int gx = 2 * x + qx, gy = 2 * y + qy, gz = 2 * z + qz;  // g1 voxel
        float g[32];
#pragma unroll
        for (int c = 0; c < 32; c++)
            g[c] = __bfloat162float(__float2bfloat16_rn(leaky(acc[c] + d.P[kOB3 + c])));
        const float sc = a.sigma ? *a.sigma : 1.0f;
        const float b = d.P[kOB4];
#pragma unroll
        for (int e = 0; e < 8; e++) {
            float yv = 0.f;
#pragma unroll
            for (int c = 0; c < 32; c++) yv = fmaf(w4[e * 32 + c], g[c], yv);
            const int ez = e >> 2, ey = (e >> 1) & 1, ex = e & 1;
            a.out.p[(long long)(2 * gz + ez) * a.out.sz + (long long)(2 * gy + ey) * a.out.sy +
                    2 * gx + ex] = sc * (yv + b);
        }
    }
};

struct OpD2 {  // g1 -> y (scaled by rms into a strided float32 volume)
    using Args = D2Args;
    static constexpr int N = 16;
    __device__ static void tile(const Args&, int& m0, int& c0, int& c1) {
        m0 = blockIdx.x * 128;
        c0 = 0;
        c1 = 1;
    }
    __device__ static void load(const Args& a, int m0, int, uint8_t* sA, uint8_t* sB, int tid) {
        const long long v = m0 + tid;
        const long long total = (long long)a.h.nx * a.h.ny * a.h.nz;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            uint4 r = zero4u();
            if (v < total) r = reinterpret_cast<const uint4*>(a.g1 + v * 32)[j];
            tc::st_vec8(sA, tid, 8 * j, r);
        }
        if (tid < 64) {
            const int d = tid >> 2, j = tid & 3;
            float w[8];
#pragma unroll
            for (int e = 0; e < 8; e++) w[e] = d < 8 ? a.P[kOW4 + d * 32 + 8 * j + e] : 0.f;
            tc::st_vec8(sB, d, 8 * j, tc::pack8(w));
        }
    }
    __device__ static void epilogue(const Args& a, int m0, int row, const float* acc) {
        const long long v = m0 + row;
        if (v >= (long long)a.h.nx * a.h.ny * a.h.nz) return;
        int x, y, z;
        decode3(v, a.h.nx, a.h.ny, x, y, z);
        const float s = a.sigma ? *a.sigma : 1.0f;
        const float b = a.P[kOB4];
#pragma unroll
        for (int d = 0; d < 8; d++) {
            const int dz = d >> 2, dy = (d >> 1) & 1, dx = d & 1;
            a.out.p[(long long)(2 * z + dz) * a.out.sz + (long long)(2 * y + dy) * a.out.sy + 2 * x +
                    dx] = s * (acc[d] + b);
        }
    }
};

// ============================================================================
// data gradients
// ============================================================================
struct OpD2d {  // gy (bf16, full grid) -> ga3 = (W4^T gy) * leaky'(a3)
    using Args = D2dArgs;
    static constexpr int N = 32;
    __device__ static void tile(const Args&, int& m0, int& c0, int& c1) {
        m0 = blockIdx.x * 128;
        c0 = 0;
        c1 = 1;
    }
    __device__ static void load(const Args& a, int m0, int, uint8_t* sA, uint8_t* sB, int tid) {
        const long long v = m0 + tid;
        const long long total = (long long)a.h.nx * a.h.ny * a.h.nz;
        float f[8];
#pragma unroll
        for (int d = 0; d < 8; d++) f[d] = 0.f;
        if (v < total) {
            int x, y, z;
            decode3(v, a.h.nx, a.h.ny, x, y, z);
            const int NX = 2 * a.h.nx, NY = 2 * a.h.ny;
#pragma unroll
            for (int d = 0; d < 8; d++) {
                const int dz = d >> 2, dy = (d >> 1) & 1, dx = d & 1;
                f[d] = __bfloat162float(
                    a.gy[((long long)(2 * z + dz) * NY + (2 * y + dy)) * NX + 2 * x + dx]);
            }
        }
        tc::st_vec8(sA, tid, 0, tc::pack8(f));
        tc::st_vec8(sA, tid, 8, zero4u());
        tc::st_vec8(sA, tid, 16, zero4u());
        tc::st_vec8(sA, tid, 24, zero4u());
        if (tid < 32) {
            float w[8];
#pragma unroll
            for (int d = 0; d < 8; d++) w[d] = a.P[kOW4 + d * 32 + tid];
            tc::st_vec8(sB, tid, 0, tc::pack8(w));
            tc::st_vec8(sB, tid, 8, zero4u());
            tc::st_vec8(sB, tid, 16, zero4u());
            tc::st_vec8(sB, tid, 24, zero4u());
        }
    }
    __device__ static void epilogue(const Args& a, int m0, int row, const float* acc) {
        const long long v = m0 + row;
        if (v >= (long long)a.h.nx * a.h.ny * a.h.nz) return;
        float f[32], g[8];
        for (int j = 0; j < 32; j += 8) {
            bf16x8_to_f(reinterpret_cast<const uint4*>(a.g1 + v * 32)[j / 8], g);
            for (int e = 0; e < 8; e++) f[j + e] = acc[j + e] * (g[e] > 0.f ? 1.0f : kSlope);
        }
        store_bf16_row(a.ga3 + v * 32, f, 32);
    }
};

struct OpD1d {  // ga3 -> glat: dlat[j] = sum_k W3[.,k,.]^T ga3[2j + k - 1]
    using Args = D1dArgs;
    static constexpr int N = 16;
    __device__ static void tile(const Args&, int& m0, int& c0, int& c1) {
        m0 = blockIdx.x * 128;
        c0 = 0;
        c1 = 64;
    }
    __device__ static void load(const Args& a, int m0, int ktap, uint8_t* sA, uint8_t* sB, int tid) {
        const long long v = m0 + tid;
        const long long total = (long long)a.l.nx * a.l.ny * a.l.nz;
        const int kz = ktap >> 4, ky = (ktap >> 2) & 3, kx = ktap & 3;
        uint4 r[4] = {zero4u(), zero4u(), zero4u(), zero4u()};
        if (v < total) {
            int x, y, z;
            decode3(v, a.l.nx, a.l.ny, x, y, z);
            const int ox = 2 * x + kx - 1, oy = 2 * y + ky - 1, oz = 2 * z + kz - 1;
            if (ox >= 0 && ox < a.h.nx && oy >= 0 && oy < a.h.ny && oz >= 0 && oz < a.h.nz) {
                const uint4* src = reinterpret_cast<const uint4*>(
                    a.ga3 + (((long long)oz * a.h.ny + oy) * a.h.nx + ox) * 32);
#pragma unroll
                for (int j = 0; j < 4; j++) r[j] = src[j];
            }
        }
#pragma unroll
        for (int j = 0; j < 4; j++) tc::st_vec8(sA, tid, 8 * j, r[j]);
        load_b(a, ktap, sB, tid);
    }
    __device__ static void load_b(const Args& a, int ktap, uint8_t* sB, int tid) {
        if (tid < 64) {
            const int i = tid >> 2, j = tid & 3;
            float w[8];
#pragma unroll
            for (int e = 0; e < 8; e++) w[e] = a.P[kOW3 + (8 * j + e) * 1024 + ktap * 16 + i];
            tc::st_vec8(sB, i, 8 * j, tc::pack8(w));
        }
    }
    __device__ static void load_async(const Args& a, int m0, int ktap, uint8_t* sA, uint8_t* sB,
                                      int tid) {
        const long long v = m0 + tid;
        const long long total = (long long)a.l.nx * a.l.ny * a.l.nz;
        const int kz = ktap >> 4, ky = (ktap >> 2) & 3, kx = ktap & 3;
        const bf16* src = a.ga3;
        bool ok = false;
        if (v < total) {
            int x, y, z;
            decode3(v, a.l.nx, a.l.ny, x, y, z);
            const int ox = 2 * x + kx - 1, oy = 2 * y + ky - 1, oz = 2 * z + kz - 1;
            if (ox >= 0 && ox < a.h.nx && oy >= 0 && oy < a.h.ny && oz >= 0 && oz < a.h.nz) {
                ok = true;
                src = a.ga3 + (((long long)oz * a.h.ny + oy) * a.h.nx + ox) * 32;
            }
        }
#pragma unroll
        for (int j = 0; j < 4; j++) tc::cp_async16(sA, tid, 8 * j, src + 8 * j, ok);
        load_b(a, ktap, sB, tid);
    }
    __device__ static void epilogue(const Args& a, int m0, int row, const float* acc) {
        const long long v = m0 + row;
        if (v >= (long long)a.l.nx * a.l.ny * a.l.nz) return;
        store_bf16_row(a.glat + v * 16, acc, 16);
    }
};

struct OpE2d {  // glat -> ga1 = (sum over taps of W2^T glat) * leaky'(a1)
    using Args = E2dArgs;
    static constexpr int N = 32;
    __device__ static void tile(const Args&, int& m0, int& c0, int& c1) {
        m0 = blockIdx.x * 128;
        c0 = 0;
        c1 = 14;  // 27 taps, two per slab, the last one padded
    }
    __device__ static void load(const Args& a, int m0, int ch, uint8_t* sA, uint8_t* sB, int tid) {
        const long long p = m0 + tid;
        const long long total = (long long)a.h.nx * a.h.ny * a.h.nz;
        int px = 0, py = 0, pz = 0;
        if (p < total) decode3(p, a.h.nx, a.h.ny, px, py, pz);
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int tap = 2 * ch + h;
            uint4 r0 = zero4u(), r1 = zero4u();
            if (p < total && tap < 27) {
                const int kz = tap / 9, ky = (tap / 3) % 3, kx = tap % 3;
                const int nz = pz + 1 - kz, ny = py + 1 - ky, nx = px + 1 - kx;
                if (nx >= 0 && ny >= 0 && nz >= 0 && !(nx & 1) && !(ny & 1) && !(nz & 1)) {
                    const int vx = nx >> 1, vy = ny >> 1, vz = nz >> 1;
                    if (vx < a.l.nx && vy < a.l.ny && vz < a.l.nz) {
                        const uint4* src = reinterpret_cast<const uint4*>(
                            a.glat + (((long long)vz * a.l.ny + vy) * a.l.nx + vx) * 16);
                        r0 = src[0];
                        r1 = src[1];
                    }
                }
            }
            tc::st_vec8(sA, tid, 16 * h, r0);
            tc::st_vec8(sA, tid, 16 * h + 8, r1);
        }
        {
            const int i = tid >> 2, j = tid & 3, h = j >> 1, o0 = (j & 1) * 8;
            const int tap = 2 * ch + h;
            float w[8];
#pragma unroll
            for (int e = 0; e < 8; e++)
                w[e] = tap < 27 ? a.P[kOW2 + (o0 + e) * 864 + tap * 32 + i] : 0.f;
            tc::st_vec8(sB, i, 8 * j, tc::pack8(w));
        }
    }
    __device__ static void epilogue(const Args& a, int m0, int row, const float* acc) {
        const long long p = m0 + row;
        if (p >= (long long)a.h.nx * a.h.ny * a.h.nz) return;
        float f[32], g[8];
        for (int j = 0; j < 32; j += 8) {
            bf16x8_to_f(reinterpret_cast<const uint4*>(a.h1 + p * 32)[j / 8], g);
            for (int e = 0; e < 8; e++) f[j + e] = acc[j + e] * (g[e] > 0.f ? 1.0f : kSlope);
        }
        store_bf16_row(a.ga1 + p * 32, f, 32);
    }
};

// ============================================================================
// weight gradients on the tensor cores (reduction over voxels, split over CTAs)
// ============================================================================
struct OpE2w {  // dW2[o][tap][i] += sum_v glat[v][o] h1[2v + tap - 1][i]
    using Args = E2wArgs;
    static constexpr int N = 16;
    __device__ static void tile(const Args& a, int& m0, int& c0, int& c1) {
        m0 = blockIdx.x * 128;  // rows r = tap * 32 + i
        const long long nv = (long long)a.l.nx * a.l.ny * a.l.nz;
        const int nch = (int)((nv + 31) / 32);
        c0 = blockIdx.y * a.chunks_per_cta;
        c1 = min(nch, c0 + a.chunks_per_cta);
        if (c1 < c0) c1 = c0;
    }
    __device__ static void load(const Args& a, int m0, int ch, uint8_t* sA, uint8_t* sB, int tid) {
        const long long nv = (long long)a.l.nx * a.l.ny * a.l.nz;
        const int vv = tid & 31, tt = tid >> 5;
        const int tap = m0 / 32 + tt;
        const long long v = (long long)ch * 32 + vv;
        float f[32];
#pragma unroll
        for (int i = 0; i < 32; i++) f[i] = 0.f;
        if (tap < 27 && v < nv) {
            int x, y, z;
            decode3(v, a.l.nx, a.l.ny, x, y, z);
            const int kz = tap / 9, ky = (tap / 3) % 3, kx = tap % 3;
            const int sx = 2 * x + kx - 1, sy = 2 * y + ky - 1, sz = 2 * z + kz - 1;
            if (sx >= 0 && sx < a.h.nx && sy >= 0 && sy < a.h.ny && sz >= 0 && sz < a.h.nz) {
                const uint4* src = reinterpret_cast<const uint4*>(
                    a.h1 + (((long long)sz * a.h.ny + sy) * a.h.nx + sx) * 32);
#pragma unroll
                for (int j = 0; j < 4; j++) bf16x8_to_f(src[j], f + 8 * j);
            }
        }
#pragma unroll
        for (int i = 0; i < 32; i++) tc::st_one(sA, tt * 32 + i, vv, __float2bfloat16_rn(f[i]));
        if (tid < 32) {
            const long long w = (long long)ch * 32 + tid;
            float g[16];
#pragma unroll
            for (int o = 0; o < 16; o++) g[o] = 0.f;
            if (w < nv) {
                const uint4* src = reinterpret_cast<const uint4*>(a.glat + w * 16);
                bf16x8_to_f(src[0], g);
                bf16x8_to_f(src[1], g + 8);
            }
#pragma unroll
            for (int o = 0; o < 16; o++) tc::st_one(sB, o, tid, __float2bfloat16_rn(g[o]));
        }
    }
    __device__ static void epilogue(const Args& a, int m0, int row, const float* acc) {
        const int r = m0 + row;
        if (r >= 27 * 32) return;
        for (int o = 0; o < 16; o++) atomicAdd(&a.grad[kOW2 + o * 864 + r], acc[o]);
    }
};

struct OpD1w {  // dW3[o][k][i] += sum_j ga3[2j + q][o] lat[j + t][i], class q = blockIdx.x
    using Args = D1wArgs;
    static constexpr int N = 32;
    __device__ static void tile(const Args& a, int& m0, int& c0, int& c1) {
        m0 = 0;  // rows r = tau * 16 + i, tau the class's 8 taps
        const long long nv = (long long)a.l.nx * a.l.ny * a.l.nz;
        const int nch = (int)((nv + 31) / 32);
        c0 = blockIdx.y * a.chunks_per_cta;
        c1 = min(nch, c0 + a.chunks_per_cta);
        if (c1 < c0) c1 = c0;
    }
    __device__ static void load(const Args& a, int, int ch, uint8_t* sA, uint8_t* sB, int tid) {
        const int q = blockIdx.x, qz = q >> 2, qy = (q >> 1) & 1, qx = q & 1;
        const long long nv = (long long)a.l.nx * a.l.ny * a.l.nz;
#pragma unroll
        for (int rep = 0; rep < 2; rep++) {
            const int idx = tid + rep * 128;
            const int vv = idx & 31, tau = idx >> 5;
            const long long j = (long long)ch * 32 + vv;
            float f[16];
#pragma unroll
            for (int i = 0; i < 16; i++) f[i] = 0.f;
            if (j < nv) {
                int x, y, z;
                decode3(j, a.l.nx, a.l.ny, x, y, z);
                int tz, kz, ty, ky, tx, kx;
                convt_tap(qz, tau >> 2, tz, kz);
                convt_tap(qy, (tau >> 1) & 1, ty, ky);
                convt_tap(qx, tau & 1, tx, kx);
                const int sx = x + tx, sy = y + ty, sz = z + tz;
                if (sx >= 0 && sx < a.l.nx && sy >= 0 && sy < a.l.ny && sz >= 0 && sz < a.l.nz) {
                    const uint4* src = reinterpret_cast<const uint4*>(
                        a.lat + (((long long)sz * a.l.ny + sy) * a.l.nx + sx) * 16);
                    bf16x8_to_f(src[0], f);
                    bf16x8_to_f(src[1], f + 8);
                }
            }
#pragma unroll
            for (int i = 0; i < 16; i++) tc::st_one(sA, tau * 16 + i, vv, __float2bfloat16_rn(f[i]));
        }
        if (tid < 32) {
            const long long j = (long long)ch * 32 + tid;
            float g[32];
#pragma unroll
            for (int o = 0; o < 32; o++) g[o] = 0.f;
            if (j < nv) {
                int x, y, z;
                decode3(j, a.l.nx, a.l.ny, x, y, z);
                const long long o = (((long long)(2 * z + qz) * a.h.ny + (2 * y + qy)) * a.h.nx +
                                     2 * x + qx);
                const uint4* src = reinterpret_cast<const uint4*>(a.ga3 + o * 32);
#pragma unroll
                for (int k = 0; k < 4; k++) bf16x8_to_f(src[k], g + 8 * k);
            }
#pragma unroll
            for (int o = 0; o < 32; o++) tc::st_one(sB, o, tid, __float2bfloat16_rn(g[o]));
        }
    }
    __device__ static void epilogue(const Args& a, int, int row, const float* acc) {
        const int q = blockIdx.x, qz = q >> 2, qy = (q >> 1) & 1, qx = q & 1;
        const int tau = row >> 4, i = row & 15;
        int tz, kz, ty, ky, tx, kx;
        convt_tap(qz, tau >> 2, tz, kz);
        convt_tap(qy, (tau >> 1) & 1, ty, ky);
        convt_tap(qx, tau & 1, tx, kx);
        const int ktap = (kz * 4 + ky) * 4 + kx;
        for (int o = 0; o < 32; o++) atomicAdd(&a.grad[kOW3 + o * 1024 + ktap * 16 + i], acc[o]);
    }
};

// ============================================================================
// CUDA-core kernels
// ============================================================================
// sum of squares of a strided volume: float partials per thread (four
// accumulators over at most a few hundred values), a block reduction in
// double, one atomic per block. A contiguous 16-byte aligned volume is read
// as one flat float4 array, four loads in flight per thread; otherwise a
// warp per row of x (float4 loads when rows are 16-byte aligned), 8 rows per
// block
__global__ void __launch_bounds__(256) k_sumsq(Vol in, double* acc) {
    const long long rows = (long long)in.ny * in.nz;
    const int lane = threadIdx.x, nx4 = in.nx >> 2;
    const bool vec = ((reinterpret_cast<uintptr_t>(in.p) & 15) == 0) && (in.sy % 4 == 0) &&
                     (in.sz % 4 == 0) && (in.nx % 4 == 0);
    const bool flat = vec && in.sy == in.nx && in.sz == (long long)in.nx * in.ny;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    if (flat) {
        const float4* p4 = reinterpret_cast<const float4*>(in.p);
        const long long n4 = rows * nx4;
        const long long step = (long long)gridDim.x * blockDim.x * blockDim.y;
        long long i = (long long)blockIdx.x * blockDim.x * blockDim.y + threadIdx.y * 32 + lane;
        for (; i + 3 * step < n4; i += 4 * step) {
            float4 v[4];
#pragma unroll
            for (int u = 0; u < 4; u++) v[u] = __ldg(p4 + i + u * step);
#pragma unroll
            for (int u = 0; u < 4; u++) {
                s0 = fmaf(v[u].x, v[u].x, s0);
                s1 = fmaf(v[u].y, v[u].y, s1);
                s2 = fmaf(v[u].z, v[u].z, s2);
                s3 = fmaf(v[u].w, v[u].w, s3);
            }
        }
        for (; i < n4; i += step) {
            const float4 v = __ldg(p4 + i);
            s0 = fmaf(v.x, v.x, s0);
            s1 = fmaf(v.y, v.y, s1);
            s2 = fmaf(v.z, v.z, s2);
            s3 = fmaf(v.w, v.w, s3);
        }
    }
    for (long long r = (long long)blockIdx.x * blockDim.y + threadIdx.y; r < rows && !flat;
         r += (long long)gridDim.x * blockDim.y) {
        const int y = (int)(r % in.ny), z = (int)(r / in.ny);
        const float* row = in.p + (long long)z * in.sz + (long long)y * in.sy;
        if (vec) {
            for (int x4 = lane; x4 < nx4; x4 += 32) {
                const float4 v = __ldg(reinterpret_cast<const float4*>(row) + x4);
                s0 = fmaf(v.x, v.x, s0);
                s1 = fmaf(v.y, v.y, s1);
                s2 = fmaf(v.z, v.z, s2);
                s3 = fmaf(v.w, v.w, s3);
            }
        } else {
            for (int x = lane; x < in.nx; x += 32) {
                const float v = __ldg(row + x);
                s0 = fmaf(v, v, s0);
            }
        }
    }
    double d = ((double)s0 + (double)s1) + ((double)s2 + (double)s3);
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    __shared__ double part[8];
    if (lane == 0) part[threadIdx.y] = d;
    __syncthreads();
    if (threadIdx.y == 0) {
        double t = lane < (int)blockDim.y ? part[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) atomicAdd(acc, t);
    }
}

__global__ void k_scale(const double* acc, long long n, float* sigma, float* inv_sigma) {
    double r = sqrt(*acc / (double)n);
    if (!(r > 0.0)) r = 1.0;
    *sigma = (float)r;
    *inv_sigma = (float)(1.0 / r);
}

// loss += mean((y - x0)^2) * scale; gy = bf16(scale * 2 (y - x0) / n); grad[b4] += sum gy
__global__ void k_loss(const float* __restrict__ y, Vol in, const float* inv_sigma, float scale,
                       bf16* gy, double* loss, float* grad) {
    const long long n = (long long)in.nx * in.ny * in.nz;
    const float s = *inv_sigma;
    double l = 0.0;
    float gsum = 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        int x, yy, z;
        decode3(i, in.nx, in.ny, x, yy, z);
        const float x0 = in.p[(long long)z * in.sz + (long long)yy * in.sy + x] * s;
        const float d = y[i] - x0;
        l += (double)d * d;
        const bf16 g = __float2bfloat16_rn(scale * 2.0f * d / (float)n);
        gy[i] = g;
        gsum += __bfloat162float(g);
    }
    for (int o = 16; o > 0; o >>= 1) {
        l += __shfl_xor_sync(0xffffffffu, l, o);
        gsum += __shfl_xor_sync(0xffffffffu, gsum, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(loss, l * scale / (double)n);
        atomicAdd(&grad[kOB4], gsum);
    }
}

// patch-conv weight gradients (rank 8) and the bias gradients:
//   dW1[c][d] += sum_v ga1[v][c] xq[2v + d],   dW4[d][i] += sum_v gy[2v + d] g1[v][i]
//   db1 += sum ga1, db2 += sum glat, db3 += sum ga3
// a warp per voxel, lane = channel: lanes 0..7 load the voxel's 8 patch
// inputs and lanes 8..15 its 8 output gradients, shared by shuffles; each
// lane accumulates its row of the two outer products; the 8 warps of a block
// are summed in shared memory and the block adds its sums with one atomic per
// output
__global__ void __launch_bounds__(256) k_small_grads(Vol in, const float* inv_sigma,
                                                     const bf16* __restrict__ ga1,
                                                     const bf16* __restrict__ gy,
                                                     const bf16* __restrict__ g1,
                                                     const bf16* __restrict__ ga3,
                                                     const bf16* __restrict__ glat, Dims3 h,
                                                     Dims3 l, float* grad) {
    constexpr int kVals = 19;  // per lane: dW1 row (8), dW4 column (8), db1, db3, db2
    __shared__ float red[8][kVals][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long long nh = (long long)h.nx * h.ny * h.nz;
    const long long nl = (long long)l.nx * l.ny * l.nz;
    const long long gw = (long long)blockIdx.x * 8 + wid, nw = (long long)gridDim.x * 8;
    const float s = *inv_sigma;
    const int NX = 2 * h.nx, NY = 2 * h.ny;
    const int e = lane & 7, ez = e >> 2, ey = (e >> 1) & 1, ex = e & 1;
    float w1[8], w4[8], b1 = 0.f, b3 = 0.f, b2 = 0.f;
#pragma unroll
    for (int d = 0; d < 8; d++) w1[d] = w4[d] = 0.f;
    for (long long v = gw; v < nh; v += nw) {
        int x, y, z;
        decode3(v, h.nx, h.ny, x, y, z);
        float mine = 0.f;
        if (lane < 8)
            mine = __bfloat162float(__float2bfloat16_rn(
                in.p[(long long)(2 * z + ez) * in.sz + (long long)(2 * y + ey) * in.sy + 2 * x + ex] *
                s));
        else if (lane < 16)
            mine = __bfloat162float(
                gy[((long long)(2 * z + ez) * NY + (2 * y + ey)) * NX + 2 * x + ex]);
        const float a = __bfloat162float(ga1[v * 32 + lane]);
        const float gg = __bfloat162float(g1[v * 32 + lane]);
        b1 += a;
        b3 += __bfloat162float(ga3[v * 32 + lane]);
#pragma unroll
        for (int d = 0; d < 8; d++) {
            w1[d] = fmaf(a, __shfl_sync(0xffffffffu, mine, d), w1[d]);
            w4[d] = fmaf(__shfl_sync(0xffffffffu, mine, 8 + d), gg, w4[d]);
        }
    }
    if (lane < 16)
        for (long long v = gw; v < nl; v += nw) b2 += __bfloat162float(glat[v * 16 + lane]);
#pragma unroll
    for (int d = 0; d < 8; d++) {
        red[wid][d][lane] = w1[d];
        red[wid][8 + d][lane] = w4[d];
    }
    red[wid][16][lane] = b1;
    red[wid][17][lane] = b3;
    red[wid][18][lane] = b2;
    __syncthreads();
    for (int k = threadIdx.x; k < kVals * 32; k += blockDim.x) {
        const int val = k >> 5, ln = k & 31;
        float t = 0.f;
#pragma unroll
        for (int w = 0; w < 8; w++) t += red[w][val][ln];
        if (val < 8)
            atomicAdd(&grad[kOW1 + ln * 8 + val], t);
        else if (val < 16)
            atomicAdd(&grad[kOW4 + (val - 8) * 32 + ln], t);
        else if (val == 16)
            atomicAdd(&grad[kOB1 + ln], t);
        else if (val == 17)
            atomicAdd(&grad[kOB3 + ln], t);
        else if (ln < 16)
            atomicAdd(&grad[kOB2 + ln], t);
    }
}

__global__ void k_sumsq_vec(const float* __restrict__ g, int n, double* out) {
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        s += (double)g[i] * g[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

// Adam with the gradient scaled to a global L2 norm of at most clip
__global__ void k_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2, const double* gnorm2, float clip) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double nrm = sqrt(*gnorm2);
    const float scale = (clip > 0.f && nrm > clip) ? (float)(clip / nrm) : 1.0f;
    const float gi = g[i] * scale;
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ============================================================================
// launchers
// ============================================================================
template <class Op>
cudaError_t run(const typename Op::Args& a, dim3 grid, int* status, cudaStream_t s) {
    tc::k_tc_gemm<Op><<<grid, 128, 0, s>>>(a, status);
    return cudaGetLastError();
}

template <class Op>
cudaError_t run_async(const typename Op::Args& a, dim3 grid, int* status, cudaStream_t s) {
    tc::k_tc_gemm_async<Op><<<grid, 128, 0, s>>>(a, status);
    return cudaGetLastError();
}

inline unsigned tiles(long long rows) { return (unsigned)((rows + 127) / 128); }

}  // namespace ae

using namespace ae;

cudaError_t ae_gemm_test(const GemmArgs& a, int N, int* status, cudaStream_t s) {
    if (N == 16) return run_async<OpGemm<16>>(a, dim3(tiles(a.M)), status, s);
    if (N == 32) return run_async<OpGemm<32>>(a, dim3(tiles(a.M)), status, s);
    return cudaErrorInvalidValue;
}

cudaError_t ae_rms(const Vol& in, AeScalars* sc, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(&sc->sumsq, 0, sizeof(double), s);
    if (e != cudaSuccess) return e;
    const long long n = (long long)in.nx * in.ny * in.nz;
    long long blocks = ((long long)in.ny * in.nz + 7) / 8;
    if (blocks > 152 * 8) blocks = 152 * 8;
    k_sumsq<<<(unsigned)blocks, dim3(32, 8), 0, s>>>(in, &sc->sumsq);
    k_scale<<<1, 1, 0, s>>>(&sc->sumsq, n, &sc->sigma, &sc->inv_sigma);
    return cudaGetLastError();
}

cudaError_t ae_encode(const float* P, const Vol& in, bf16* h1, bf16* lat, AeScalars* sc,
                      float* sigma_out, int* status, cudaStream_t s, bool keep_h1,
                      bool sumsq_ready) {
    cudaError_t e = cudaSuccess;
    if (sumsq_ready) {
        k_scale<<<1, 1, 0, s>>>(&sc->sumsq, (long long)in.nx * in.ny * in.nz, &sc->sigma,
                                &sc->inv_sigma);
        e = cudaGetLastError();
    } else {
        e = ae_rms(in, sc, s);
    }
    if (e != cudaSuccess) return e;
    const Dims3 h{in.nx / 2, in.ny / 2, in.nz / 2}, l{in.nx / 4, in.ny / 4, in.nz / 4};
    e = keep_h1 ? cudaErrorNotSupported : ae_encode_march(P, in, &sc->inv_sigma, lat, status, s);
    if (e == cudaErrorNotSupported) {
        cudaGetLastError();
        E1Args a1{in, &sc->inv_sigma, P, h1, h};
        e = run<OpE1>(a1, dim3(tiles((long long)h.nx * h.ny * h.nz)), status, s);
        if (e != cudaSuccess) return e;
        E2Args a2{h1, h, P, lat, l};
        e = run_async<OpE2>(a2, dim3(tiles((long long)l.nx * l.ny * l.nz)), status, s);
    }
    if (e != cudaSuccess) return e;
    if (sigma_out) e = cudaMemcpyAsync(sigma_out, &sc->sigma, sizeof(float),
                                       cudaMemcpyDeviceToDevice, s);
    return e;
}

cudaError_t ae_decode(const float* P, const bf16* lat, const float* sigma, const Vol& out, bf16* g1,
                      int* status, cudaStream_t s) {
    const Dims3 h{out.nx / 2, out.ny / 2, out.nz / 2}, l{out.nx / 4, out.ny / 4, out.nz / 4};
    if (g1) {  // two passes through g1 (training keeps g1 for the backward pass)
        D1Args a1{lat, l, P, g1, h};
        cudaError_t e =
            run_async<OpD1>(a1, dim3(tiles((long long)l.nx * l.ny * l.nz), 8), status, s);
        if (e != cudaSuccess) return e;
        D2Args a2{g1, h, P, sigma, out};
        return run<OpD2>(a2, dim3(tiles((long long)h.nx * h.ny * h.nz)), status, s);
    }
    D12Args a{D1Args{lat, l, P, nullptr, h}, sigma, out};
    const cudaError_t e = ae_decode_march(a, status, s);
    if (e != cudaErrorNotSupported) return e;
    cudaGetLastError();
    return run_async<OpD12>(a, dim3(tiles((long long)l.nx * l.ny * l.nz), 8), status, s);
}

// loss and gradient of one sample, accumulated into grad (scale = 1 / batch)
cudaError_t ae_sample_grad(const float* P, const Vol& in, float scale, const AeTrainBufs& b,
                           AeScalars* sc, double* loss, float* grad, int* status, cudaStream_t s) {
    const Dims3 h{in.nx / 2, in.ny / 2, in.nz / 2}, l{in.nx / 4, in.ny / 4, in.nz / 4};
    const long long nh = (long long)h.nx * h.ny * h.nz, nl = (long long)l.nx * l.ny * l.nz;
    const long long n = (long long)in.nx * in.ny * in.nz;
    cudaError_t e = ae_encode(P, in, b.h1, b.lat, sc, nullptr, status, s, true);
    if (e != cudaSuccess) return e;
    const Vol yv{b.y, (long long)in.nx, (long long)in.nx * in.ny, in.nx, in.ny, in.nz};
    e = ae_decode(P, b.lat, nullptr, yv, b.g1, status, s);
    if (e != cudaSuccess) return e;
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    k_loss<<<(unsigned)blocks, 256, 0, s>>>(b.y, in, &sc->inv_sigma, scale, b.gy, loss, grad);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    D2dArgs d2{b.gy, h, b.g1, P, b.ga3};
    if ((e = run<OpD2d>(d2, dim3(tiles(nh)), status, s)) != cudaSuccess) return e;
    const int nch_l = (int)((nl + 31) / 32);
    const int cpc_l = max(1, (nch_l + 151) / 152);
    D1wArgs w3{b.lat, l, b.ga3, h, grad, cpc_l};
    if ((e = run<OpD1w>(w3, dim3(8, (nch_l + cpc_l - 1) / cpc_l), status, s)) != cudaSuccess)
        return e;
    D1dArgs d1{b.ga3, h, l, P, b.glat};
    if ((e = run_async<OpD1d>(d1, dim3(tiles(nl)), status, s)) != cudaSuccess) return e;
    E2wArgs w2{b.h1, h, b.glat, l, grad, cpc_l};
    if ((e = run<OpE2w>(w2, dim3(7, (nch_l + cpc_l - 1) / cpc_l), status, s)) != cudaSuccess)
        return e;
    E2dArgs d0{b.glat, l, b.h1, h, P, b.ga1};
    if ((e = run<OpE2d>(d0, dim3(tiles(nh)), status, s)) != cudaSuccess) return e;
    long long sb = (nh + 8 * 64 - 1) / (8 * 64);  // at least 64 voxels per warp
    if (sb < 1) sb = 1;
    if (sb > 152 * 4) sb = 152 * 4;
    k_small_grads<<<(unsigned)sb, 256, 0, s>>>(in, &sc->inv_sigma, b.ga1, b.gy, b.g1, b.ga3,
                                               b.glat, h, l, grad);
    return cudaGetLastError();
}

cudaError_t ae_adam(float* P, float* m, float* v, const float* g, int step, float lr, float clip,
                    double* scratch, cudaStream_t s) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(double), s);
    if (e != cudaSuccess) return e;
    k_sumsq_vec<<<64, 256, 0, s>>>(g, kNParams, scratch);
    k_adam<<<(kNParams + 255) / 256, 256, 0, s>>>(P, m, v, g, kNParams, lr, b1, b2, eps, c1, c2,
                                                  scratch, clip);
    return cudaGetLastError();
}

}  // namespace rtm
