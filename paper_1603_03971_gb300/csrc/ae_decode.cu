// Inference decoder, z-marching: D1 (transposed conv 16 -> 32, kernel 4,
// stride 2, padding 1) + LeakyReLU + D2 (transposed patch conv 32 -> 1) in one
// persistent kernel, one CTA per SM.
//
// Work item: a column of 8 x 16 latent voxels (x, y) over a range of z. For
// each latent plane z the 128 voxels of the column are the M = 128 rows of
// the 8 parities x 8 taps of D1 (K = 16 input channels each, N = 32 output
// channels), accumulated per parity into tensor memory: 52 tcgen05.mma,
// since in all but the first tap group the two parities of an x pair that
// read the window at x offset 0 share one N = 64 MMA.
//
// The A operands are never gathered. TMA copies each latent plane of the
// column with a one-voxel halo (10 x 18 voxels, zeros outside the grid) into
// a shared-memory ring as two 8-channel halves of [18][10] 16-byte rows: that
// is the canonical K-major no-swizzle layout of a 128-row operand whose 8-row
// groups are y rows (stride 160 B) and whose two K core matrices are the two
// channel halves. The operand of a tap (tz, ty, tx) is the same layout
// started at plane z + tz, row (1 + ty), column (1 + tx): a descriptor with a
// shifted start address.
//
// Roles: warp 9 (one thread) issues the TMA plane loads, each as soon as its
// ring slot is free; warp 8 (one thread) the MMAs into one of two
// accumulator buffers (2 x 256 columns);
// warpgroup 0 finishes even planes, warpgroup 1 odd planes, four parities at
// a time: tcgen05.ld of their accumulators (one row per thread),
// LeakyReLU(acc + b3) rounded to bfloat16 (as the training decoder rounds
// g1) into four 128 x 32 K-major A operands in shared memory, then one
// thread issues D2 as tensor-core products, [128 x 32] g1 x [32 x 16] W4
// (rows 8..15 zero), into the accumulator columns just drained; the 8 results
// per parity are read back, scaled by the snapshot's rms and stored as the
// float4 rows of the latent voxel's 4 x 4 x 4 output block. mbarriers: plane
// full (TMA bytes), plane free (commit of the last MMAs that read it),
// accumulator full (commit), accumulator free (128 epilogue arrivals), D2
// done (commit). Every wait is bounded and shares an abort flag; the
// warpgroups vote on each wait's outcome, so they leave together.

#include <cuda.h>
#include <cuda_bf16.h>
#include <string.h>

#include <algorithm>

#include "ae_internal.h"
#include "packed_f32x2.cuh"
#include "tc_gemm.cuh"
#include "tma_encode.h"
#include "wait_clock.cuh"

namespace rtm {
namespace ae {
namespace {

constexpr int TX = 8, TY = 16;                 // latent column (128 MMA rows)
constexpr int HX = TX + 2, HY = TY + 2;        // with the halo
constexpr int kHalfBytes = 2944;               // one 8-channel half plane (2880 B, 128-aligned)
constexpr int kPlaneBytes = 2 * kHalfBytes;
constexpr int kTmaBytes = 2 * HX * HY * 16;    // bytes one plane load delivers
constexpr int kSlots = 9;                      // plane ring
constexpr int kW3Bytes = 64 * 1024;            // 64 B operands (parity, tap): 32 x 16, 1 KB each
constexpr int kA2Bytes = 128 * 32 * 2;          // D2 A operand: 128 rows x 32 channels, bf16
// W3 operands, plane ring, b3 (128 B), the D2 B operand W4 (16 x 32 bf16,
// 1 KB), four D2 A operands per epilogue warpgroup: > half an SM, 1 CTA
constexpr int kSmem = 128 + kW3Bytes + kSlots * kPlaneBytes + 128 + 1024 + 2 * 4 * kA2Bytes;
constexpr int kTmemCols = 512;
constexpr int kThreads = 320;
constexpr long long kLimit = 1LL << 24;
constexpr uint32_t kSuspendNs = 20000;  // longest sleep of one poll (woken by the phase)

struct Sched {
    int ncx, ncy, nzc, zc, nitems;
};

__device__ __forceinline__ void item_coords(const Sched& S, int lnz, int item, int& cx, int& cy,
                                            int& z0, int& nz) {
    cx = item % S.ncx;
    cy = (item / S.ncx) % S.ncy;
    const int kz = item / (S.ncx * S.ncy);
    z0 = kz * S.zc;
    nz = min(S.zc, lnz - z0);
}

// taps of a transposed conv (kernel 4, stride 2, padding 1) along one axis
// for output parity q: tap tau reads input i + t with kernel index k
__device__ __forceinline__ void taps(int q, int tau, int& t, int& k) {
    if (q == 0) {
        t = tau ? -1 : 0;
        k = tau ? 3 : 1;
    } else {
        t = tau ? 0 : 1;
        k = tau ? 2 : 0;
    }
}

static_assert(kSlope > 0.f && kSlope < 1.f, "LeakyReLU as a maximum needs 0 < slope < 1");

// KB block of the B operand of (parity q, tap tau) in the W3 table: per
// x-parity pair m = q >> 1 and tap group g = tau >> 1 (z, y tap bits), four
// blocks [q1 tap x 0, q0 tap x 0, q1 tap x 1, q0 tap x 1] (q0 = 2 m,
// q1 = 2 m + 1), so that q0's x-offset-0 tap (x tap 0) and q1's (x tap 1)
// are one 64-row operand
__host__ __device__ constexpr int w3_block(int q, int tau) {
    return (q >> 1) * 16 + (tau >> 1) * 4 + (tau & 1) * 2 + (1 - (q & 1));
}

__device__ __forceinline__ void bar_expect(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(b)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(b)) : "memory");
}
// bounded wait; gives up early once another thread has raised the abort flag
__device__ __forceinline__ bool wait_bar(uint64_t* b, uint32_t parity, volatile int* abort_flag) {
    const uint32_t a = tc::smem_u32(b);
    if (mbar_try_wait_sleep(a, parity, kSuspendNs)) return true;
    const unsigned long long t0 = wait_now();
    for (long long i = 0; i < kLimit; i++) {
        if (mbar_try_wait_sleep(a, parity, kSuspendNs)) return true;
        if (abort_flag && *abort_flag) return false;
        if (wait_expired(i, t0)) break;
    }
    if (abort_flag) *abort_flag = 1;
    return false;
}
__device__ __forceinline__ void tma_plane(uint8_t* dst, const CUtensorMap* map, int kc, int x, int y,
                                          int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(tc::smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(kc), "r"(x), "r"(y), "r"(z),
        "r"(tc::smem_u32(bar))
        : "memory");
}
// 16 columns of this warp's lanes into r, without waiting: the registers
// must not be read before a tmem_wait_regs16 that names them
__device__ __forceinline__ void tmem_ld16_nw(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}
// wait for this thread's TMEM loads; the 16 registers are operands, so no
// read of them can be scheduled before the wait
__device__ __forceinline__ void tmem_wait_regs16(uint32_t* r) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                   "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                   "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
                 :
                 : "memory");
}
// all 128 threads of a warpgroup (named barrier id) agree: true only if v is
// true in every one of them; also a barrier of the warpgroup
__device__ __forceinline__ bool wg_all(bool v, int id) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, %2, 128, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id)
        : "memory");
    return r != 0;
}
// 8 columns of this warp's lanes into r, without waiting (as tmem_ld16_nw)
__device__ __forceinline__ void tmem_ld8_nw(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7])
        : "r"(taddr)
        : "memory");
}

// byte offset of (row o, k) in a 32 x 16 K-major operand (LBO 128, SBO 256)
__device__ __forceinline__ int b_off(int o, int k) {
    return (o >> 3) * 256 + (k >> 3) * 128 + (o & 7) * 16 + (k & 7) * 2;
}

__global__ void __launch_bounds__(kThreads, 1)
    k_decode_march(const __grid_constant__ D12Args A, const __grid_constant__ CUtensorMap map,
                   const Sched S, int* status) {
    extern __shared__ uint8_t dsm_raw[];
    __shared__ __align__(8) uint64_t full[kSlots], freed[kSlots], acc_full[2], acc_free[2], fin,
        d2_full[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;

    uint8_t* base = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(dsm_raw) + 127) & ~static_cast<uintptr_t>(127));
    uint8_t* w3 = base;
    uint8_t* ring = base + kW3Bytes;
    float* b3s = reinterpret_cast<float*>(ring + kSlots * kPlaneBytes);  // b3[32]
    uint8_t* b4t = ring + kSlots * kPlaneBytes + 128;  // W4 as a 16 x 32 K-major operand
    uint8_t* a2 = b4t + 1024;                          // D2 A operands

    const D1Args& d = A.d1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int* abrt = &abort_flag;

    if (tid == 0) {
        for (int s = 0; s < kSlots; s++) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&freed[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            tc::mbar_init(&acc_full[b], 1);
            tc::mbar_init(&acc_free[b], 128);
            tc::mbar_init(&d2_full[b], 1);
        }
        tc::mbar_init(&fin, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tc::tmem_alloc(&tmem_slot, kTmemCols);
    // B operands: (parity q, tap tau) -> W3[o][kz][ky][kx][i] as a 32 x 16 K-major tile
    for (int idx = tid; idx < 64 * 32 * 2; idx += kThreads) {
        const int j = idx & 1, o = (idx >> 1) & 31, t = idx >> 6, q = t >> 3, tau = t & 7;
        int tz, kz, ty, ky, tx, kx;
        taps(q >> 2, tau >> 2, tz, kz);
        taps((q >> 1) & 1, (tau >> 1) & 1, ty, ky);
        taps(q & 1, tau & 1, tx, kx);
        const int ktap = (kz * 4 + ky) * 4 + kx;
        float w[8];
#pragma unroll
        for (int e = 0; e < 8; e++) w[e] = d.P[kOW3 + o * 1024 + ktap * 16 + 8 * j + e];
        *reinterpret_cast<uint4*>(w3 + w3_block(q, tau) * 1024 + b_off(o, 8 * j)) =
            tc::pack8(w);
    }
    // W4[e][c] (e = (ez, ey, ex), c = channel) as rows e of a 16 x 32 K-major
    // bf16 operand, rows 8..15 zero
    for (int idx = tid; idx < 16 * 4; idx += kThreads) {
        const int e = idx >> 2, c8 = (idx & 3) * 8;
        float w[8];
#pragma unroll
        for (int i = 0; i < 8; i++) w[i] = e < 8 ? d.P[kOW4 + e * 32 + c8 + i] : 0.f;
        tc::st_vec8(b4t, e, c8, tc::pack8(w));
    }
    if (tid < 32) b3s[tid] = d.P[kOB3 + tid];
    tc::fence_proxy_async();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const int lnx = d.l.nx, lny = d.l.ny, lnz = d.l.nz;

    if (warp == 8) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            constexpr uint32_t idesc = tc::idesc_bf16(128, 32), idesc64 = tc::idesc_bf16(128, 64);
            const uint32_t ring_a = tc::smem_u32(ring);
            const uint64_t dB0 = tc::sdesc(tc::smem_u32(w3), 128, 256);
            int out = 0, base_seq = 0;
            bool ok = true;
            for (int item = blockIdx.x; item < S.nitems && ok; item += gridDim.x) {
                int cx, cy, z0, nz;
                item_coords(S, lnz, item, cx, cy, z0, nz);
                for (int zi = 0; zi < nz && ok; zi++) {
                    for (int s = base_seq + zi; s <= base_seq + zi + 2 && ok; s++)
                        ok = wait_bar(&full[s % kSlots], (uint32_t)((s / kSlots) & 1), abrt);
                    const int b = out & 1, u = out >> 1;
                    if (ok && u >= 1) ok = wait_bar(&acc_free[b], (uint32_t)((u - 1) & 1), abrt);
                    if (!ok) break;
                    tc::tc_fence_after();
                    // descriptors: the start-address field is address >> 4 and no
                    // operand crosses 256 KB, so offsets add to the field directly
                    uint64_t dA[3];
#pragma unroll
                    for (int t = 0; t < 3; t++)
                        dA[t] = tc::sdesc(ring_a + ((base_seq + zi + t) % kSlots) * kPlaneBytes,
                                          kHalfBytes, HX * 16);
                    // opaque per plane, so that the 64 B descriptors are not hoisted
                    // out of the loop into registers
                    uint64_t dB;
                    asm volatile("mov.b64 %0, %1;" : "=l"(dB) : "l"(dB0));
                    // per x-parity pair (q0 = 2 m, q1 = 2 m + 1) and tap group
                    // (tz', ty'): q0 reads x offsets 0 (x tap 0) and -1 (x tap 1),
                    // q1 reads +1 (x tap 0) and 0 (x tap 1). In every group but
                    // the first the two x-offset-0 taps are one N = 64 MMA into
                    // both parities' columns, issued between q1's x tap 0 and
                    // q0's x tap 1, so every parity sums its taps in tap order;
                    // the first group runs as four MMAs, the first of each
                    // parity overwriting its accumulator. 52 MMAs per plane
#pragma unroll
                    for (int m = 0; m < 4; m++) {
                        const uint32_t c0 = tmem + b * 256 + (2 * m) * 32, c1 = c0 + 32;
#pragma unroll
                        for (int g = 0; g < 4; g++) {
                            int tz, kz, ty, ky;
                            taps(m >> 1, g >> 1, tz, kz);
                            taps(m & 1, g & 1, ty, ky);
                            const uint64_t a = dA[1 + tz] + (uint64_t)((1 + ty) * HX);
                            const uint64_t bg = dB + (uint64_t)((m * 16 + g * 4) * 64);
                            if (g == 0) {
                                tc::mma_bf16(c0, a + 1, bg + 64, idesc, 0u);       // q0, x tap 0
                                tc::mma_bf16(c0, a + 0, bg + 3 * 64, idesc, 1u);   // q0, x tap 1
                                tc::mma_bf16(c1, a + 2, bg, idesc, 0u);            // q1, x tap 0
                                tc::mma_bf16(c1, a + 1, bg + 2 * 64, idesc, 1u);   // q1, x tap 1
                            } else {
                                tc::mma_bf16(c1, a + 2, bg, idesc, 1u);            // q1, x tap 0
                                tc::mma_bf16(c0, a + 1, bg + 64, idesc64, 1u);     // both, offset 0
                                tc::mma_bf16(c0, a + 0, bg + 3 * 64, idesc, 1u);   // q0, x tap 1
                            }
                        }
                    }
                    tc::mma_commit(&acc_full[b]);
                    // plane z - 1 is read by no later output of this item
                    tc::mma_commit(&freed[(base_seq + zi) % kSlots]);
                    if (zi == nz - 1) {
                        tc::mma_commit(&freed[(base_seq + zi + 1) % kSlots]);
                        tc::mma_commit(&freed[(base_seq + zi + 2) % kSlots]);
                    }
                    out++;
                }
                base_seq += nz + 2;
            }
            if (!ok) *abrt = 1;
            tc::mma_commit(&fin);
            if (!wait_bar(&fin, 0, nullptr)) *abrt = 1;
        }
    } else if (warp == 9) {
        if (lane == 0) {
            // ---------------- plane loader ----------------
            // every latent plane of every item (with its z halo) into the next
            // ring slot as soon as the MMAs that read the slot last are done
            int l_seq = 0;
            bool ok = true;
            for (int item = blockIdx.x; item < S.nitems && ok; item += gridDim.x) {
                int lcx, lcy, lz0, lnzi;
                item_coords(S, lnz, item, lcx, lcy, lz0, lnzi);
                for (int l_j = 0; l_j < lnzi + 2; l_j++, l_seq++) {
                    const int slot = l_seq % kSlots;
                    if (l_seq >= kSlots)
                        ok = wait_bar(&freed[slot], (uint32_t)((l_seq / kSlots - 1) & 1), abrt);
                    if (!ok) break;
                    bar_expect(&full[slot], kTmaBytes);
                    uint8_t* dst = ring + slot * kPlaneBytes;
                    for (int kc = 0; kc < 2; kc++)
                        tma_plane(dst + kc * kHalfBytes, &map, kc, lcx * TX - 1, lcy * TY - 1,
                                  lz0 - 1 + l_j, &full[slot]);
                }
            }
            // every copy must land before the CTA leaves (after an abort some
            // were never waited for): wait, bounded and ignoring the flag, for
            // each slot's last load; a completed one answers at once
            for (int q = (l_seq > kSlots ? l_seq - kSlots : 0); q < l_seq; q++)
                wait_bar(&full[q % kSlots], (uint32_t)((q / kSlots) & 1), nullptr);
        }
    } else {
        // ---------------- epilogue warpgroups ----------------
        const int g = warp >> 2, row = tid & 127, ly = row >> 3, lx = row & 7;
        const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
        const float b4 = d.P[kOB4];
        const float sc = A.sigma ? *A.sigma : 1.0f;
        const bool vec = ((reinterpret_cast<uintptr_t>(A.out.p) & 15) == 0) &&
                         (A.out.sy % 4 == 0) && (A.out.sz % 4 == 0);
        // b3 as packed pairs and the slope as a pair (f32x2 arithmetic, IEEE
        // single precision per lane)
        uint64_t b3p[16];
#pragma unroll
        for (int c = 0; c < 16; c++) b3p[c] = f32x2::pack(b3s[2 * c], b3s[2 * c + 1]);
        const uint64_t slope2 = f32x2::pack(kSlope, kSlope);
        uint8_t* atile = a2 + g * 4 * kA2Bytes;  // this warpgroup's four D2 A operands
        constexpr uint32_t idesc2 = tc::idesc_bf16(128, 16);
        int out = 0, d2_phase = 0;
        bool ok = true, d2_pending = false;
        for (int item = blockIdx.x; item < S.nitems && ok; item += gridDim.x) {
            int cx, cy, z0, nz;
            item_coords(S, lnz, item, cx, cy, z0, nz);
            const int X = cx * TX + lx, Y = cy * TY + ly;
            const bool valid = X < lnx && Y < lny;
            for (int zi = 0; zi < nz; zi++, out++) {
                if ((out & 1) != g) continue;
                const int u = out >> 1;
                ok = wg_all(wait_bar(&acc_full[g], (uint32_t)(u & 1), abrt), 1 + g);
                if (!ok) break;
                tc::tc_fence_after();
                const int Z = z0 + zi;
                const uint32_t tb = lane_base + g * 256;
#pragma unroll 1
                for (int qz = 0; qz < 2 && ok; qz++) {
                    // g1 = bf16(LeakyReLU(acc + b3)) of the four parities (qz, qy, qx)
                    // into the A operands (row = latent voxel, K = channel), one
                    // parity's TMEM load in flight while the one before it is
                    // processed; LeakyReLU as max(h, slope h) on packed pairs (the
                    // same bits as the select form for 0 < slope < 1)
                    auto tile = [&](int p4, const uint32_t* r) {
                        uint8_t* t = atile + p4 * kA2Bytes;
#pragma unroll
                        for (int k8 = 0; k8 < 4; k8++) {
                            uint32_t w[4];
#pragma unroll
                            for (int c = 0; c < 4; c++) {
                                const int i = 8 * k8 + 2 * c;
                                const uint64_t h = f32x2::add(
                                    f32x2::pack(__uint_as_float(r[i]), __uint_as_float(r[i + 1])),
                                    b3p[i >> 1]);
                                const uint64_t sh = f32x2::mul(h, slope2);
                                float h0, h1, s0, s1;
                                f32x2::unpack(h, h0, h1);
                                f32x2::unpack(sh, s0, s1);
                                w[c] = tc::pack2(fmaxf(h0, s0), fmaxf(h1, s1));
                            }
                            tc::st_vec8(t, row, 8 * k8, make_uint4(w[0], w[1], w[2], w[3]));
                        }
                    };
                    const uint32_t cq = tb + qz * 4 * 32;
                    uint32_t x0[32], x1[32];
                    tmem_ld16_nw(cq, x0);
                    tmem_ld16_nw(cq + 16, x0 + 16);
                    tmem_wait_regs16(x0);
                    tmem_wait_regs16(x0 + 16);
                    tmem_ld16_nw(cq + 32, x1);
                    tmem_ld16_nw(cq + 48, x1 + 16);
                    tile(0, x0);
                    tmem_wait_regs16(x1);
                    tmem_wait_regs16(x1 + 16);
                    tmem_ld16_nw(cq + 64, x0);
                    tmem_ld16_nw(cq + 80, x0 + 16);
                    tile(1, x1);
                    tmem_wait_regs16(x0);
                    tmem_wait_regs16(x0 + 16);
                    tmem_ld16_nw(cq + 96, x1);
                    tmem_ld16_nw(cq + 112, x1 + 16);
                    tile(2, x0);
                    tmem_wait_regs16(x1);
                    tmem_wait_regs16(x1 + 16);
                    tile(3, x1);
                    // the generic-proxy tile writes and the drained accumulator
                    // columns, then one thread issues the D2 products into those
                    // columns: [128 x 32] g1 x [32 x 16] W4 (rows 8..15 zero)
                    tc::fence_proxy_async();
                    tc::tc_fence_before();
                    asm volatile("bar.sync %0, 128;" ::"r"(1 + g) : "memory");
                    if (row == 0) {
                        tc::tc_fence_after();
                        const uint64_t dB = tc::sdesc(tc::smem_u32(b4t), 128, 512);
#pragma unroll
                        for (int p = 0; p < 4; p++) {
                            const uint64_t dA =
                                tc::sdesc(tc::smem_u32(atile + p * kA2Bytes), 128, 512);
                            const uint32_t dcol = tmem + g * 256 + (qz * 4 + p) * 32;
                            tc::mma_bf16(dcol, dA, dB, idesc2, 0u);
                            tc::mma_bf16(dcol, dA + 16, dB + 16, idesc2, 1u);  // K 16..31
                        }
                        tc::mma_commit(&d2_full[g]);
                        d2_pending = true;
                    }
                    // (the vote also orders the next half's tile writes after
                    // every thread's wait: the products have read the tiles)
                    ok = wg_all(wait_bar(&d2_full[g], (uint32_t)(d2_phase & 1), abrt), 1 + g);
                    if (!ok) break;
                    d2_phase++;
                    if (row == 0) d2_pending = false;
                    tc::tc_fence_after();
                    uint32_t ry[32];
#pragma unroll
                    for (int p = 0; p < 4; p++) tmem_ld8_nw(tb + (qz * 4 + p) * 32, ry + 8 * p);
                    tmem_wait_regs16(ry);
                    tmem_wait_regs16(ry + 16);
                    float y[4][8];
#pragma unroll
                    for (int p = 0; p < 4; p++)
#pragma unroll
                        for (int i = 0; i < 8; i++) y[p][i] = __uint_as_float(ry[8 * p + i]);
                    if (valid) {
#pragma unroll
                        for (int qy = 0; qy < 2; qy++) {
#pragma unroll
                            for (int ezy = 0; ezy < 4; ezy++) {
                                const int ez = ezy >> 1, ey = ezy & 1;
                                // x: (qx, ex) = (0, 0), (0, 1), (1, 0), (1, 1)
                                const float* ya = y[qy * 2];
                                const float* yb = y[qy * 2 + 1];
                                float* o = A.out.p + (long long)(4 * Z + 2 * qz + ez) * A.out.sz +
                                           (long long)(4 * Y + 2 * qy + ey) * A.out.sy + 4 * X;
                                const float4 v = make_float4(
                                    sc * (ya[ezy * 2] + b4), sc * (ya[ezy * 2 + 1] + b4),
                                    sc * (yb[ezy * 2] + b4), sc * (yb[ezy * 2 + 1] + b4));
                                if (vec) {
                                    *reinterpret_cast<float4*>(o) = v;
                                } else {
                                    o[0] = v.x;
                                    o[1] = v.y;
                                    o[2] = v.z;
                                    o[3] = v.w;
                                }
                            }
                        }
                    }
                }
                if (!ok) break;
                tc::tc_fence_before();
                bar_arrive(&acc_free[g]);
            }
        }
        // products still in flight must complete before the tensor memory is freed
        if (d2_pending) wait_bar(&d2_full[g], (uint32_t)(d2_phase & 1), nullptr);
    }
    tc::tc_fence_before();
    __syncthreads();
    if (tid == 0 && *abrt && status) atomicCAS(status, 0, tc::kErrTimeout);
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, kTmemCols);
    }
}

// decoder choice: 0 auto (z-marching kernel when TMA is available), 1 the
// GEMM-engine decoder, 2 the z-marching kernel
int g_decoder = 0;

}  // namespace
}  // namespace ae

void ae_set_decoder(int which) { ae::g_decoder = which; }

// Returns cudaErrorNotSupported when the z-marching kernel cannot run (no
// tensor-map encoder, misaligned latent, or not selected): the caller then
// uses the GEMM-engine decoder.
cudaError_t ae_decode_march(const ae::D12Args& a, int* status, cudaStream_t s) {
    using namespace ae;
    if (g_decoder == 1) return cudaErrorNotSupported;
    EncodeTiledFn enc = tma_encoder();
    if (!enc || (reinterpret_cast<uintptr_t>(a.d1.lat) & 15)) return cudaErrorNotSupported;
    static int nsm = 0;
    if (nsm == 0) {
        cudaError_t e = cudaFuncSetAttribute(k_decode_march,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
        if (e != cudaSuccess) return e;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (nsm < 1) nsm = 1;
    }
    const Dims3 l = a.d1.l;
    CUtensorMap map;
    memset(&map, 0, sizeof map);
    const cuuint64_t dims[5] = {8, 2, (cuuint64_t)l.nx, (cuuint64_t)l.ny, (cuuint64_t)l.nz};
    const cuuint64_t strides[4] = {16, 32, 32ull * l.nx, 32ull * l.nx * l.ny};
    const cuuint32_t box[5] = {8, 1, HX, HY, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<bf16*>(a.d1.lat), dims, strides,
            box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorNotSupported;
    // z chunk: smallest per-CTA makespan, counting each chunk's two halo
    // planes as one plane of work
    Sched S;
    S.ncx = (l.nx + TX - 1) / TX;
    S.ncy = (l.ny + TY - 1) / TY;
    const long long ncol = (long long)S.ncx * S.ncy;
    long long best = -1;
    S.zc = l.nz;
    for (int zc = std::min(4, l.nz); zc <= l.nz; zc++) {
        const long long items = ncol * ((l.nz + zc - 1) / zc);
        const long long span = (items + nsm - 1) / nsm * (zc + 1);
        if (best < 0 || span < best) {
            best = span;
            S.zc = zc;
        }
    }
    S.nzc = (l.nz + S.zc - 1) / S.zc;
    S.nitems = (int)(ncol * S.nzc);
    const int grid = std::min(nsm, S.nitems);
    k_decode_march<<<grid, kThreads, kSmem, s>>>(a, map, S, status);
    return cudaGetLastError();
}

}  // namespace rtm
