// Stencil step with TMA plane loads (tuning variants 2 and 3).
//
// The same leapfrog update and epilogues as k_stencil, with the plane loads
// moved to the tensor memory accelerator. A block owns a tile of x-y columns
// and marches a z slab. Variant 2: 256-thread blocks, 64 x 16 tiles at
// radius 4 (four points per thread) and 32 x 16 at radius 8 (two points per
// thread). Variant 3: 128-thread blocks, 64 x 8 tiles with four points per
// thread at both radii. One thread issues
// 3D bulk tensor copies of the next planes into shared-memory rings, P
// planes ahead of the one being computed, each slot completed on its
// mbarrier by the copy's transaction bytes (expect-tx):
//  - joint ring (radius-4 forward modes): R + P + 1 planes of u^n with the
//    r-wide halo, the newest being the queue head, and P + 1 planes of the
//    pointwise operands (u^{n-1}, c);
//  - split ring (radius 8, radius-4 backward modes): the P + 1 centre planes
//    of u^n with halo, while the queue head (plane z + r, no halo) travels
//    with the pointwise operands (u^{n-1}, c, and the snapshot / accumulator
//    of the backward modes). Cells outside the padded grid arrive as zeros:
//    the Dirichlet ghost cells.
// Each thread keeps the 2r + 1 column values of its points in a register
// queue along z, moved once per G planes, and reads its x-y neighbours from
// the centre plane in shared memory. One block barrier per plane frees the
// slots for refilling.
//
// Tensor-map rules respected here: every row starts on a 16-byte boundary
// (NX % 4 == 0), the x coordinate of every copy is a multiple of 4 floats
// (x0 and x0 - r with x0 a multiple of 4: the tile width times the block
// index, plus the launch region's x origin, which is rounded down to a
// multiple of 4, and r % 4 == 0), boxes are at most 256 per side and their
// rows a multiple of 16 bytes, and shared destinations are 128-byte aligned.
// Copies only load; negative or out-of-range coordinates read zeros.

#include <cuda.h>
#include <string.h>

#include <mutex>

#include "../../include/rtm.h"
#include "packed_f32x2.cuh"
#include "rtm_internal.h"
#include "stencil_common.cuh"
#include "tma_encode.h"
#include "wait_clock.cuh"

namespace rtm {

namespace {

constexpr long long kTmaWaitLimit = 1LL << 26;

struct TmaMaps {
    CUtensorMap u, prev, c, e1, e2, uh;  // uh: u^n without halo (queue heads)
};

// V consecutive x points per thread: 4 (16-byte vectors), except in the
// 16-row tiles at radius 8, whose 256-thread blocks hold 2 (the 2r + G deep
// register queue of 4-point vectors would allow one block per SM). The 8-row
// radius-8 tiles keep 4 points per thread: 128 registers, four blocks of 128
// threads per SM, and half the per-plane overhead and shared-memory x loads
// per point
template <int R, int BY = 16>
__host__ __device__ constexpr int points_per_thread() {
    return (R == 8 && BY == 16) ? 2 : 4;
}

// tile: 16 threads along x (V floats each) by BYT rows, one row per thread
// (16 rows: 256 threads, the default; 8 rows: 128 threads, more blocks per SM
// and twice the y halo per row, an autotuner choice)
template <int R, int V, int BYT = 16>
struct TmaTile {
    static constexpr int BX = 16;          // threads along x, V floats each
    static constexpr int BY = BYT;         // threads along y
    static constexpr int TX = V * BX;      // floats
    static constexpr int TY = BY;          // rows
    static constexpr int SW = TX + 2 * R;  // shared row width (floats)
    static constexpr int SH = TY + 2 * R;  // shared rows
    static constexpr int HX = R / V;       // halo vectors per side per row
    static_assert(R % 4 == 0 && R % V == 0, "radius must be a multiple of 4 and of V");
    static_assert(BY == 16 || BY == 8, "16- or 8-row tiles");
};

template <int V>
struct Vec {
    float v[V];
};
template <int V>
__device__ __forceinline__ Vec<V> vzero() {
    Vec<V> r;
#pragma unroll
    for (int i = 0; i < V; i++) r.v[i] = 0.f;
    return r;
}
template <int V>
__device__ __forceinline__ Vec<V> vlds(const float* p) {  // shared memory
    Vec<V> r;
    if constexpr (V == 4) {
        const float4 t = *reinterpret_cast<const float4*>(p);
        r.v[0] = t.x, r.v[1] = t.y, r.v[2] = t.z, r.v[3] = t.w;
    } else {
        const float2 t = *reinterpret_cast<const float2*>(p);
        r.v[0] = t.x, r.v[1] = t.y;
    }
    return r;
}
template <int V>
__device__ __forceinline__ Vec<V> vld_keep(const float* p) {  // read-only global, keep cached
    Vec<V> r;
    if constexpr (V == 4) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(p));
        r.v[0] = t.x, r.v[1] = t.y, r.v[2] = t.z, r.v[3] = t.w;
    } else {
        const float2 t = __ldg(reinterpret_cast<const float2*>(p));
        r.v[0] = t.x, r.v[1] = t.y;
    }
    return r;
}
template <int V>
__device__ __forceinline__ void vst_stream(float* p, const Vec<V>& a) {
    if constexpr (V == 4)
        __stcs(reinterpret_cast<float4*>(p), make_float4(a.v[0], a.v[1], a.v[2], a.v[3]));
    else
        __stcs(reinterpret_cast<float2*>(p), make_float2(a.v[0], a.v[1]));
}

// the Laplacian on packed pairs of points, with half the floating-point
// instructions. Radius 4 keeps the scalar form's order of sums (two point
// pairs per thread already give two independent chains); radius 8 (one pair
// per thread, eight offsets) sums even and odd offsets separately and then
// adds, halving the dependent chain
template <int R>
__host__ __device__ constexpr bool packed_math() {
    return true;
}
template <int R>
__host__ __device__ constexpr bool split_chains() {
    return R == 8;
}

template <int MODE>
__host__ __device__ constexpr int aux_planes() {
    return (MODE == MODE_BWD_IMAGE || MODE == MODE_BWD_GRAD) ? 4 : 2;
}

// u^n ring layout. Joint: the ring holds planes z .. z + r + P with their
// halo; plane z + r is the queue head, and it stays in the ring until it is
// the centre plane. Split (radius 8): the ring holds only the P + 1 centre
// planes with their halo, and the queue head (plane z + r, the tile without
// halo) travels with the pointwise operands of plane z: each plane is copied
// twice from L2, but the ring shrinks from 2r + P + 1 halo planes (66 KB at
// radius 8) to P + 1 (18 KB), so three blocks fit per SM in every mode
template <int R, int MODE>
__host__ __device__ constexpr bool split_ring() {
    return R == 8 || aux_planes<MODE>() == 4;
}

// planes loaded ahead of the one being computed
template <int R, int MODE>
__host__ __device__ constexpr int tma_prefetch() {
    return (R == 4 && aux_planes<MODE>() == 4) ? 1 : 2;
}

// the register queue moves once per G planes (2r + G entries, the plane body
// unrolled G times): 2r / G vector moves per plane instead of 2r. 576^3,
// radius 8, 2-point vectors: G = 1 / 2 / 4 gave 204.8 / 210.6 / 215.8
// Gpoint-updates/s; radius 4: G = 1 / 2 gave 318.4 / 320.8 (G = 3 spills
// under the 80-register cap of three blocks per SM). Radius 8 with 4-point
// vectors keeps G = 2 (the queue is 72 registers)
template <int R, int V>
__host__ __device__ constexpr int queue_group() {
    return (R == 8 && V == 2) ? 4 : 2;
}

template <int R, int MODE, int BY = 16>
struct TmaCfg {
    using T = TmaTile<R, points_per_thread<R, BY>(), BY>;
    static constexpr bool SPLIT = split_ring<R, MODE>();
    static constexpr int NA = aux_planes<MODE>();
    static constexpr int NAH = NA + (SPLIT ? 1 : 0);  // aux ring entries per plane
    static constexpr int P = tma_prefetch<R, MODE>();
    static constexpr int SU = SPLIT ? P + 1 : R + P + 1;
    static constexpr int SA = P + 1;
    static constexpr int UPLANE = T::SH * T::SW;  // floats
    static constexpr int APLANE = T::TY * T::TX;
    static constexpr int SMEM = (SU * UPLANE + SA * NAH * APLANE) * 4;
};

__device__ __forceinline__ uint32_t s_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void bar_init(uint64_t* b) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_u32(b)));
}
__device__ __forceinline__ void bar_expect(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_u32(b)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool bar_poll(uint32_t a, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    return done != 0;
}
// bounded wait (poll count and elapsed time); false if it ran out (then the
// block's abort flag is raised) or if the block aborted while it waited. The
// caller reads the abort flag once per plane, before its waits: a completed
// phase answers the first poll without a shared-memory read of the flag
__device__ __forceinline__ bool bar_wait(uint64_t* b, uint32_t parity, int* abort_flag) {
    const uint32_t a = s_u32(b);
    if (bar_poll(a, parity)) return true;  // the common case: the plane is in
    const unsigned long long t0 = wait_now();
    for (long long i = 0; i < kTmaWaitLimit; i++) {
        if (bar_poll(a, parity)) return true;
        if (*reinterpret_cast<volatile int*>(abort_flag)) return false;
        if (wait_expired(i, t0)) break;
    }
    *reinterpret_cast<volatile int*>(abort_flag) = 1;
    return false;
}
// bounded wait that ignores the abort flag: lets a copy already in flight
// land in shared memory before the block leaves
__device__ __forceinline__ void bar_drain(uint64_t* b, uint32_t parity) {
    const uint32_t a = s_u32(b);
    const unsigned long long t0 = wait_now();
    for (long long i = 0; i < kTmaWaitLimit; i++)
        if (bar_poll(a, parity) || wait_expired(i, t0)) return;
}
__device__ __forceinline__ void tma3(float* dst, const CUtensorMap* map, int x, int y, int z,
                                     uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(s_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(s_u32(bar))
        : "memory");
}

// resident blocks per SM. 16-row tiles: three 256-thread blocks, registers
// capped at 80 per thread; at radius 4 the forward modes need 73 KB of shared
// memory, the split-ring backward modes 54 KB; at radius 8 the split ring
// needs 36-48 KB. 8-row tiles (128 threads): five blocks at radius 4 (102
// registers, 17-29 KB), four at radius 8 (128 registers, 4-point vectors,
// 30-53 KB)
template <int R, int MODE, int BY = 16>
constexpr int tma_min_blocks() {
    return BY == 16 ? 3 : (R == 8 ? 4 : 5);
}
// the rings of the resident blocks fit the SM's 228 KB (1 KB reserved per block)
template <int R, int MODE, int BY = 16>
constexpr bool rings_fit() {
    return tma_min_blocks<R, MODE, BY>() * (TmaCfg<R, MODE, BY>::SMEM + 1024 + 256) <=
           228 * 1024;
}

// STALL: the instance that takes a test-armed stall (rtm_set_test_stall);
// compiled only for the forward step with 8-row tiles, so that no other
// instance carries its code
template <int R, int MODE, int BY, bool STALL = false>
__global__ void __launch_bounds__(16 * BY, (tma_min_blocks<R, MODE, BY>()))
    k_stencil_tma(const __grid_constant__ StepArgs A, const __grid_constant__ TmaMaps M, int* status,
                  int stall) {
    constexpr int V = points_per_thread<R, BY>();
    using T = TmaTile<R, V, BY>;
    using VT = Vec<V>;
    using C = TmaCfg<R, MODE, BY>;
    constexpr int NA = C::NA;
    extern __shared__ __align__(128) float dsm[];
    float* uring = dsm;
    float* aring = dsm + C::SU * C::UPLANE;
    __shared__ __align__(8) uint64_t ubar[C::SU];
    __shared__ __align__(8) uint64_t abar[C::SA];
    __shared__ int abort_flag;

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * T::BX + tx;
    const int x0 = A.xorg + blockIdx.x * T::TX, y0 = A.yorg + blockIdx.y * T::TY;
    const int x = x0 + V * tx, y = y0 + ty;
    const int zb = A.zorg + blockIdx.z * A.zchunk;
    const int ze = min(A.zend, zb + A.zchunk);
    // cells this thread updates: inside the array and the launch region (a
    // vector straddling the region's x end is computed whole; a launch over
    // one subdomain of a decomposed grid leaves its halo columns and rows
    // untouched: their end is a multiple of V)
    const int xend_v = (A.xend + V - 1) / V * V;
    const bool own = x < A.NX && y < A.NY && x < xend_v && y < A.yend;
    const size_t plane = (size_t)A.NX * (size_t)A.NY;
    const size_t col = (size_t)y * A.NX + x;
    const bool xm = (x + V - 1 >= A.nb) && (x < A.nb + A.nx);
    const bool ym = (y >= A.nb) && (y < A.nb + A.ny);
    const size_t slab_col = (size_t)(y - A.nb) * A.NX + x;
    const size_t slab_plane = (size_t)A.ny * A.NX;
    // reverse mode: all of this thread's cells lie in the model's x-y range
    const bool model_col = x >= A.nb && x + V - 1 < A.nb + A.nx && y >= A.nb && y < A.nb + A.ny;

    if (tid == 0) {
        for (int s = 0; s < C::SU; s++) bar_init(&ubar[s]);
        for (int s = 0; s < C::SA; s++) bar_init(&abar[s]);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // newest u^n plane copied with its halo: the queue head of the last step
    // (joint ring) or the last centre plane (split ring)
    const int last_u = C::SPLIT ? ze - 1 : ze - 1 + R;
    // thread 0 issues planes in order: u^n planes [zb, u_end), pointwise
    // operand planes [zb, a_end)
    int u_end = zb, a_end = zb;
    auto issue_u = [&](int p) {
        u_end = p + 1;
        const int slot = (p - zb) % C::SU;
        bar_expect(&ubar[slot], C::UPLANE * 4);
        tma3(uring + slot * C::UPLANE, &M.u, x0 - R, y0 - R, p, &ubar[slot]);
    };
    auto issue_a = [&](int p) {
        a_end = p + 1;
        const int slot = (p - zb) % C::SA;
        float* base = aring + slot * C::NAH * C::APLANE;
        uint32_t extra = 0;
        if constexpr (STALL) {
            // block 0's copy of the plane `stall` planes before its last
            // expects 16 bytes that never arrive, so the wait for it runs
            // out. No later copy reuses that slot, so no wait can take a
            // later phase of its mbarrier for the stuck one
            if (p == ze - 1 - stall && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0)
                extra = 16;
        }
        bar_expect(&abar[slot], C::NAH * C::APLANE * 4 + extra);
        tma3(base, &M.prev, x0, y0, p, &abar[slot]);
        tma3(base + C::APLANE, &M.c, x0, y0, p, &abar[slot]);
        if constexpr (C::SPLIT) tma3(base + NA * C::APLANE, &M.uh, x0, y0, p + R, &abar[slot]);
        if constexpr (MODE == MODE_BWD_IMAGE) {
            if (A.snap_padded)
                tma3(base + 2 * C::APLANE, &M.e1, x0, y0, p, &abar[slot]);
            else
                tma3(base + 2 * C::APLANE, &M.e1, x0, y0 - A.nb, p - A.nb, &abar[slot]);
            tma3(base + 3 * C::APLANE, &M.e2, x0, y0 - A.nb, p - A.nb, &abar[slot]);
        } else if constexpr (MODE == MODE_BWD_GRAD) {
            tma3(base + 2 * C::APLANE, &M.e1, x0, y0, p, &abar[slot]);
            tma3(base + 3 * C::APLANE, &M.e2, x0, y0, p, &abar[slot]);
        }
    };
    if (tid == 0) {
        for (int p = zb; p < zb + (C::SPLIT ? 0 : R) + C::P && p <= last_u; p++) issue_u(p);
        for (int p = zb; p < zb + C::P && p < ze; p++) issue_a(p);
    }

    VT gxy = vzero<V>();
    if (own) {
        const float gyv = A.gy[y];
#pragma unroll
        for (int i = 0; i < V; i++) gxy.v[i] = A.gx[x + i] * gyv;
    }
    // queue planes zb - R .. zb + R - 1 straight from global memory
    // queue: plane z0 + t of a group reads entries t .. t + 2r (head 2r + t)
    constexpr int G = queue_group<R, V>();
    VT q[2 * R + G];
#pragma unroll
    for (int i = 0; i < 2 * R; i++) {
        const int zz = zb - R + i;
        q[i] = (own && zz >= 0 && zz < A.NZ) ? vld_keep<V>(A.u_cur + (size_t)zz * plane + col)
                                             : vzero<V>();
    }
#pragma unroll
    for (int i = 2 * R; i < 2 * R + G; i++) q[i] = vzero<V>();

    const int own_off = (R + ty) * T::SW + R + V * tx;  // this vector in a u^n plane
    const int aux_off = ty * T::TX + V * tx;             // this vector in an aux plane

    float ssq = 0.f;  // MODE_FWD_SUMSQ: this thread's share of the sum of squares
    // ring slots and mbarrier phases, advanced by counting
    int sc = 0, pc = 0;                          // centre plane z
    int shd = R % C::SU, phd = (R / C::SU) & 1;  // queue head plane z + R
    int sa = 0, pa = 0;                          // pointwise operands of plane z
    for (int z0 = zb; z0 < ze; z0 += G) {
#pragma unroll
    for (int t = 0; t < G; t++) {
        const int z = z0 + t;
        if (z >= ze) break;  // the same for every thread of the block
        if (tid == 0 && !abort_flag) {
            const int pu = z + (C::SPLIT ? 0 : R) + C::P;
            if (pu <= last_u) issue_u(pu);
            if (z + C::P < ze) issue_a(z + C::P);
        }
        bool ok = !*reinterpret_cast<volatile int*>(&abort_flag);  // once per plane
        if constexpr (!C::SPLIT) {
            ok = ok && bar_wait(&ubar[shd], (uint32_t)phd, &abort_flag);
            q[2 * R + t] = vlds<V>(uring + shd * C::UPLANE + own_off);
        }
        ok = ok && bar_wait(&ubar[sc], (uint32_t)pc, &abort_flag);
        ok = ok && bar_wait(&abar[sa], (uint32_t)pa, &abort_flag);
        const float* S = uring + sc * C::UPLANE;
        const float* aux = aring + sa * C::NAH * C::APLANE;
        if constexpr (C::SPLIT) q[2 * R + t] = vlds<V>(aux + NA * C::APLANE + aux_off);

        if (own && ok) {
            float v[V + 2 * R];
#pragma unroll
            for (int h = 0; h < T::HX; h++) {
                const VT l = vlds<V>(S + (R + ty) * T::SW + V * tx + V * h);
                const VT r = vlds<V>(S + (R + ty) * T::SW + R + V * tx + V + V * h);
#pragma unroll
                for (int i = 0; i < V; i++) {
                    v[V * h + i] = l.v[i];
                    v[R + V + V * h + i] = r.v[i];
                }
            }
#pragma unroll
            for (int i = 0; i < V; i++) v[R + i] = q[R + t].v[i];
            VT lap;
            if constexpr (packed_math<R>()) {
                uint64_t L2[V / 2], L2o[V / 2];
                const uint64_t a0 = f32x2::pack(A.a[0], A.a[0]);
#pragma unroll
                for (int j = 0; j < V / 2; j++) {
                    L2[j] = f32x2::mul(a0, f32x2::pack(q[R + t].v[2 * j], q[R + t].v[2 * j + 1]));
                    L2o[j] = 0;  // the bit pattern of two +0.0f
                }
#pragma unroll
                for (int k = 1; k <= R; k++) {
                    const VT ym_ = vlds<V>(S + (R + ty - k) * T::SW + R + V * tx);
                    const VT yp_ = vlds<V>(S + (R + ty + k) * T::SW + R + V * tx);
                    const uint64_t ak = f32x2::pack(A.a[k], A.a[k]);
#pragma unroll
                    for (int j = 0; j < V / 2; j++) {
                        const int i = 2 * j;
                        const uint64_t px = f32x2::add(f32x2::pack(v[R + i - k], v[R + i + 1 - k]),
                                                 f32x2::pack(v[R + i + k], v[R + i + 1 + k]));
                        const uint64_t py = f32x2::add(f32x2::pack(ym_.v[i], ym_.v[i + 1]),
                                                 f32x2::pack(yp_.v[i], yp_.v[i + 1]));
                        const uint64_t pz = f32x2::add(f32x2::pack(q[R + t - k].v[i], q[R + t - k].v[i + 1]),
                                                 f32x2::pack(q[R + t + k].v[i], q[R + t + k].v[i + 1]));
                        if (split_chains<R>() && (k & 1))
                            L2o[j] = f32x2::fma(ak, f32x2::add(f32x2::add(px, py), pz), L2o[j]);
                        else
                            L2[j] = f32x2::fma(ak, f32x2::add(f32x2::add(px, py), pz), L2[j]);
                    }
                }
#pragma unroll
                for (int j = 0; j < V / 2; j++) {
                    if constexpr (split_chains<R>())
                        f32x2::unpack(f32x2::add(L2[j], L2o[j]), lap.v[2 * j], lap.v[2 * j + 1]);
                    else
                        f32x2::unpack(L2[j], lap.v[2 * j], lap.v[2 * j + 1]);
                }
            } else {
#pragma unroll
                for (int i = 0; i < V; i++) lap.v[i] = A.a[0] * q[R + t].v[i];
#pragma unroll
                for (int k = 1; k <= R; k++) {
                    const VT ym_ = vlds<V>(S + (R + ty - k) * T::SW + R + V * tx);
                    const VT yp_ = vlds<V>(S + (R + ty + k) * T::SW + R + V * tx);
#pragma unroll
                    for (int i = 0; i < V; i++) {
                        const float px = v[R + i - k] + v[R + i + k];
                        const float py = ym_.v[i] + yp_.v[i];
                        const float pz = q[R + t - k].v[i] + q[R + t + k].v[i];
                        lap.v[i] = fmaf(A.a[k], (px + py) + pz, lap.v[i]);
                    }
                }
            }
            const VT up = vlds<V>(aux + aux_off);
            const VT cc = vlds<V>(aux + C::APLANE + aux_off);
            const float gzv = A.gz[z];
            const VT& qc = q[R + t];
            VT out;
            if constexpr (MODE == MODE_REV) {
                // the sponge factor is 1 in the model region: the forward
                // update with the two time levels swapped
#pragma unroll
                for (int i = 0; i < V; i++) out.v[i] = fmaf(cc.v[i], lap.v[i], 2.0f * qc.v[i]) - up.v[i];
                if (!model_col) {  // cells outside the model keep their value
#pragma unroll
                    for (int i = 0; i < V; i++) {
                        const int mx = x + i - A.nb, my = y - A.nb;
                        if (mx < 0 || mx >= A.nx || my < 0 || my >= A.ny) out.v[i] = up.v[i];
                    }
                }
            } else {
#pragma unroll
                for (int i = 0; i < V; i++) {
                    const float g = gxy.v[i] * gzv;
                    out.v[i] = g * fmaf(cc.v[i], lap.v[i], 2.0f * qc.v[i]) - (g * g) * up.v[i];
                }
            }
            const size_t o = (size_t)z * plane + col;
            vst_stream<V>(A.u_prev + o, out);
            if constexpr (MODE == MODE_FWD_SUMSQ) {
                if (ym && z >= A.nb && z < A.nb + A.nz) {
#pragma unroll
                    for (int i = 0; i < V; i++)
                        if (x + i >= A.nb && x + i < A.nb + A.nx) ssq = fmaf(out.v[i], out.v[i], ssq);
                }
            } else if constexpr (MODE == MODE_FWD_SNAP) {
                if (xm && ym && z >= A.nb && z < A.nb + A.nz)
                    vst_stream<V>(A.snap + (size_t)(z - A.nb) * slab_plane + slab_col, out);
            } else if constexpr (MODE == MODE_BWD_IMAGE) {
                if (xm && ym && z >= A.nb && z < A.nb + A.nz) {
                    const VT sv = vlds<V>(aux + 2 * C::APLANE + aux_off);
                    VT acc = vlds<V>(aux + 3 * C::APLANE + aux_off);
#pragma unroll
                    for (int i = 0; i < V; i++) acc.v[i] = fmaf(sv.v[i], out.v[i], acc.v[i]);
                    vst_stream<V>(A.acc + (size_t)(z - A.nb) * slab_plane + slab_col, acc);
                }
            } else if constexpr (MODE == MODE_FWD_LU) {
                vst_stream<V>(A.snap + o, lap);
            } else if constexpr (MODE == MODE_BWD_GRAD) {
                const VT sv = vlds<V>(aux + 2 * C::APLANE + aux_off);
                VT acc = vlds<V>(aux + 3 * C::APLANE + aux_off);
#pragma unroll
                for (int i = 0; i < V; i++) acc.v[i] = fmaf(out.v[i], sv.v[i], acc.v[i]);
                vst_stream<V>(A.acc + o, acc);
            }
        }
        __syncthreads();  // every thread is done with planes z (centre, aux): slots reusable
        if (++sc == C::SU) sc = 0, pc ^= 1;
        if (++shd == C::SU) shd = 0, phd ^= 1;
        if (++sa == C::SA) sa = 0, pa ^= 1;
    }
#pragma unroll
        for (int i = 0; i < 2 * R; i++) q[i] = q[i + G];
    }
    if constexpr (MODE == MODE_FWD_SUMSQ) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ssq += __shfl_xor_sync(0xffffffffu, ssq, o);
        if ((tid & 31) == 0 && ssq != 0.f) atomicAdd(A.sumsq, (double)ssq);
    }
    // every copy must land before the block exits: a slab shorter than r
    // issued planes [ze, zb + r) that no step waited for, and after an abort
    // the remaining waits returned at once. The newest plane issued into each
    // slot is the only one that can still be in flight (an earlier one was
    // waited for before its slot was refilled), so wait for it, bounded and
    // ignoring the abort flag; a completed phase answers at once
    if (tid == 0) {
        for (int s = 0; s < C::SU; s++) {
            const int j = u_end - 1 - zb;
            if (j < s) break;
            const int jl = s + (j - s) / C::SU * C::SU;
            bar_drain(&ubar[s], (uint32_t)((jl / C::SU) & 1));
        }
        for (int s = 0; s < C::SA; s++) {
            const int j = a_end - 1 - zb;
            if (j < s) break;
            const int jl = s + (j - s) / C::SA * C::SA;
            bar_drain(&abar[s], (uint32_t)((jl / C::SA) & 1));
        }
        if (abort_flag && status) atomicCAS(status, 0, 5);  // RTM_ERR_TIMEOUT
    }
}

// ---- host side: tensor maps ---------------------------------------------------
cudaError_t encode_map(CUtensorMap* m, const float* base, int nx, int ny, int nz, int bx,
                       int by);

// A shot launches the stencil thousands of times on the same few buffers, so
// the encoded maps are kept per thread, keyed by every encoding argument, and
// reused (least recently encoded entry replaced)
struct MapKey {
    const float* base;
    int nx, ny, nz, bx, by;
    bool operator==(const MapKey& o) const {
        return base == o.base && nx == o.nx && ny == o.ny && nz == o.nz && bx == o.bx &&
               by == o.by;
    }
};
constexpr int kMapCache = 64;
struct MapCache {
    MapKey key[kMapCache];
    CUtensorMap map[kMapCache];
    int n = 0, next = 0;
};
thread_local MapCache t_maps;

cudaError_t make_map(CUtensorMap* m, const float* base, int nx, int ny, int nz, int bx, int by) {
    const MapKey k{base, nx, ny, nz, bx, by};
    MapCache& c = t_maps;
    for (int i = 0; i < c.n; i++)
        if (c.key[i] == k) {
            *m = c.map[i];
            return cudaSuccess;
        }
    cudaError_t e = encode_map(m, base, nx, ny, nz, bx, by);
    if (e != cudaSuccess) return e;
    int slot;
    if (c.n < kMapCache) {
        slot = c.n++;
    } else {
        slot = c.next;
        c.next = (c.next + 1) % kMapCache;
    }
    c.key[slot] = k;
    c.map[slot] = *m;
    return cudaSuccess;
}

cudaError_t encode_map(CUtensorMap* m, const float* base, int nx, int ny, int nz, int bx,
                       int by) {
    EncodeTiledFn f = tma_encoder();
    if (!f) return cudaErrorNotSupported;
    if (((uintptr_t)base % 16) || (nx % 4)) return cudaErrorInvalidValue;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t strides[2] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = f(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides,
                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// dynamic shared memory and carveout of a TMA stencil instance
template <class K>
cudaError_t set_tma_attrs(K kernel, int smem) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                cudaSharedmemCarveoutMaxShared);
}

template <int R, int MODE, int BY>
cudaError_t launch_tma_t(const StepArgs& a, int* status, cudaStream_t s) {
    using T = TmaTile<R, points_per_thread<R, BY>(), BY>;
    constexpr int smem = TmaCfg<R, MODE, BY>::SMEM;
    static_assert(rings_fit<R, MODE, BY>(), "rings do not fit the resident blocks");
    static bool attr = false;
    if (!attr) {
        cudaError_t e = set_tma_attrs(k_stencil_tma<R, MODE, BY>, smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    TmaMaps M;
    memset(&M, 0, sizeof M);
    cudaError_t e;
    if ((e = make_map(&M.u, a.u_cur, a.NX, a.NY, a.NZ, T::TX + 2 * R, T::TY + 2 * R)) != cudaSuccess)
        return e;
    if ((e = make_map(&M.prev, a.u_prev, a.NX, a.NY, a.NZ, T::TX, T::TY)) != cudaSuccess) return e;
    if (TmaCfg<R, MODE, BY>::SPLIT &&
        (e = make_map(&M.uh, a.u_cur, a.NX, a.NY, a.NZ, T::TX, T::TY)) != cudaSuccess)
        return e;
    if ((e = make_map(&M.c, a.c, a.NX, a.NY, a.NZ, T::TX, T::TY)) != cudaSuccess) return e;
    if (MODE == MODE_BWD_IMAGE) {
        if ((e = a.snap_padded ? make_map(&M.e1, a.snap, a.NX, a.NY, a.NZ, T::TX, T::TY)
                               : make_map(&M.e1, a.snap, a.NX, a.ny, a.nz, T::TX, T::TY)) !=
            cudaSuccess)
            return e;
        if ((e = make_map(&M.e2, a.acc, a.NX, a.ny, a.nz, T::TX, T::TY)) != cudaSuccess) return e;
    } else if (MODE == MODE_BWD_GRAD) {
        if ((e = make_map(&M.e1, a.snap, a.NX, a.NY, a.NZ, T::TX, T::TY)) != cudaSuccess) return e;
        if ((e = make_map(&M.e2, a.acc, a.NX, a.NY, a.NZ, T::TX, T::TY)) != cudaSuccess) return e;
    }
    dim3 block(T::BX, T::BY);
    dim3 grid((a.xend - a.xorg + T::TX - 1) / T::TX, (a.yend - a.yorg + T::TY - 1) / T::TY,
              (a.zend - a.zorg + a.zchunk - 1) / a.zchunk);
    if (a.xorg % 4 || a.xend <= a.xorg || a.yend <= a.yorg || a.zend <= a.zorg)
        return cudaErrorInvalidValue;
    if constexpr (MODE == MODE_FWD && BY == 8) {
        const int stall = take_test_stall(RTM_STALL_STENCIL);
        if (stall >= 0) {
            static bool attr_stall = false;
            if (!attr_stall) {
                cudaError_t e = set_tma_attrs(k_stencil_tma<R, MODE, BY, true>, smem);
                if (e != cudaSuccess) return e;
                attr_stall = true;
            }
            k_stencil_tma<R, MODE, BY, true><<<grid, block, smem, s>>>(a, M, status, stall);
            return cudaGetLastError();
        }
    }
    k_stencil_tma<R, MODE, BY><<<grid, block, smem, s>>>(a, M, status, -1);
    return cudaGetLastError();
}

template <int R, int BY>
cudaError_t launch_tma_r(int mode, const StepArgs& a, int* status, cudaStream_t s) {
    switch (mode) {
        case MODE_FWD: return launch_tma_t<R, MODE_FWD, BY>(a, status, s);
        case MODE_FWD_SNAP: return launch_tma_t<R, MODE_FWD_SNAP, BY>(a, status, s);
        case MODE_BWD_IMAGE: return launch_tma_t<R, MODE_BWD_IMAGE, BY>(a, status, s);
        case MODE_FWD_LU: return launch_tma_t<R, MODE_FWD_LU, BY>(a, status, s);
        case MODE_BWD_GRAD: return launch_tma_t<R, MODE_BWD_GRAD, BY>(a, status, s);
        case MODE_REV: return launch_tma_t<R, MODE_REV, BY>(a, status, s);
        case MODE_FWD_SUMSQ: return launch_tma_t<R, MODE_FWD_SUMSQ, BY>(a, status, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

EncodeTiledFn tma_encoder() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

bool tma_available() { return tma_encoder() != nullptr; }

cudaError_t launch_stencil_tma(int radius, int mode, const StepArgs& a, int* status,
                               cudaStream_t s, int tile_rows) {
    if (a.zchunk < 1 || (tile_rows != 16 && tile_rows != 8)) return cudaErrorInvalidValue;
    if (tile_rows == 8) {
        switch (radius) {
            case 4: return launch_tma_r<4, 8>(mode, a, status, s);
            case 8: return launch_tma_r<8, 8>(mode, a, status, s);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (radius) {
        case 4: return launch_tma_r<4, 16>(mode, a, status, s);
        case 8: return launch_tma_r<8, 16>(mode, a, status, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rtm
