// Inference encoder, z-marching: E1 (patch conv 1 -> 32, kernel 2, stride 2)
// + LeakyReLU + E2 (conv 32 -> 16, kernel 3, stride 2, padding 1) in one
// persistent kernel, one CTA per SM. The 32-channel intermediate h1 never
// leaves shared memory.
//
// Work item: a column of 8 x 16 latent voxels (x, y) over a range of latent
// planes z. Latent plane z reads h1 planes 2z - 1, 2z, 2z + 1; each h1 plane
// of the column is a 17 x 33 tile (one h1 voxel of halo on the low side)
// computed from two snapshot planes, which TMA copies (40 x 66 floats, zeros
// outside the volume) into a four-slot ring.
//
// E1 runs on the tensor cores as well: for each h1 plane, the warpgroup that
// owns it (warpgroup 1 even planes, warpgroup 2 odd ones; three snapshot
// slots, so that a warpgroup's next copy overlaps its current plane) writes
// the bf16(s / rms) values of every h1 voxel's 2 x 2 x 2 patch as one row of
// a 648-row A tile, the issuing thread runs 5 tcgen05.mma (M = 128 voxels,
// N = 32, K = 16: the 8 patch values, then 8 columns multiplied by the zero
// half of W1) into that warpgroup's 160 TMEM columns, and the warpgroup adds
// b1, applies LeakyReLU, rounds to bf16 and stores h1 into a three-slot ring
// laid out as E2's A operand in the canonical K-major no-swizzle layout:
// four 8-channel core-matrix columns (leading byte offset 8976 B) of
// [33][17] 16-byte rows, with the x positions split by parity (9 even, then
// 8 odd) so that every tap of the stride-2 convolution reads 8 consecutive
// rows: tap (kz, ky, kx) of latent row (ly, lx) is h1 row 2 ly + ky, slot lx
// (kx = 0), 9 + lx (kx = 1) or lx + 1 (kx = 2); 8-row groups (one per ly)
// are 544 B apart. The products, sums and rounding points are those of the
// GEMM-engine encoder, so the latents are the same.
//
// E2 runs on the tensor cores, one h1 plane at a time: as soon as plane p is
// complete, one thread issues its 9 taps x 2 tcgen05.mma (M = 128 latent
// voxels, N = 16, K = 16 channels) into the accumulator of every latent plane
// that reads it (plane 2m: kz = 2 of latent m - 1, then kz = 0 of latent m;
// plane 2m + 1: kz = 1 of latent m), so each latent sums its 27 taps in the
// order of the GEMM-engine encoder and each h1 slot is freed after one use.
// Two 16-column accumulators alternate between latent planes; warpgroup 3
// adds b2, rounds to bf16 and stores the latent rows. The issuing thread runs
// an event loop of non-blocking mbarrier tests (snapshot slot free -> next
// copy; A tile built -> E1 MMAs; h1 plane complete and accumulator free ->
// its E2 MMAs). mbarriers: snapshot full (TMA bytes) / free (128 arrivals),
// A tile full (128 arrivals) / E1 done (commit), h1 full (128 arrivals) /
// free (commit), accumulator full (commit) / free (128 arrivals). Every wait
// is bounded and shares an abort flag.

#include <cuda.h>
#include <cuda_bf16.h>
#include <string.h>

#include <algorithm>

#include "ae_internal.h"
#include "tc_gemm.cuh"
#include "tma_encode.h"
#include "wait_clock.cuh"

namespace rtm {
namespace ae {
namespace {

constexpr int TX = 8, TY = 16;          // latent column (128 MMA rows)
constexpr int HX = 2 * TX + 1;          // h1 tile: 17 x 33
constexpr int HY = 2 * TY + 1;
constexpr int NVOX = HX * HY;           // 561
constexpr int kRowBytes = HX * 16;      // one h1 row of one 8-channel column: 272 B
constexpr int kKcBytes = HY * kRowBytes;                 // 8976 B
constexpr int kH1Bytes = 35968;                          // 4 columns (35904 B), 128-aligned
constexpr int SX = 40, SYR = 2 * HY;                     // snapshot box: 40 x 66 x 2
constexpr int kSnapBytes = SX * SYR * 2 * 4;             // 21120
constexpr int kW2Bytes = 54 * 512;                       // 27 taps x 2 halves of 16 x 16
constexpr int kSS = 3, kSH = 3;
constexpr int kLook = 3;  // snapshot loads ahead of the next h1 plane to multiply
constexpr long long kIdleLimit = 1LL << 26;  // producer loop turns without progress
constexpr int kW1Bytes = 1024;      // W1 as a 32 x 16 operand (k 8..15 zero)
constexpr int kARows = 648;         // E1 A tile: 5 M tiles of 128 rows + 8 rows read as K half 2
constexpr int kATileBytes = kARows * 16;                 // 10368
constexpr int kE1Col = 32;          // E1 accumulators: 2 x (5 x 32) TMEM columns from here
constexpr int kSmem = 128 + kW2Bytes + kW1Bytes + kSS * kSnapBytes + kSH * kH1Bytes +
                      2 * kATileBytes;
constexpr int kThreads = 13 * 32;
constexpr int kTmemCols = 512;
constexpr long long kLimit = 1LL << 24;

struct Sched {
    int ncx, ncy, zc, nitems;
};

struct EncArgs {
    const float* P;
    const float* inv_sigma;
    bf16* lat;
    Dims3 l, h;
};

__device__ __forceinline__ void item_coords(const Sched& S, int lnz, int item, int& cx, int& cy,
                                            int& z0, int& nz) {
    cx = item % S.ncx;
    cy = (item / S.ncx) % S.ncy;
    z0 = (item / (S.ncx * S.ncy)) * S.zc;
    nz = min(S.zc, lnz - z0);
}

__device__ __forceinline__ float lrelu(float a) { return a > 0.f ? a : kSlope * a; }

__device__ __forceinline__ void bar_expect(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(b)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool wait_bar(uint64_t* b, uint32_t parity, volatile int* abort_flag) {
    const uint32_t a = tc::smem_u32(b);
    const unsigned long long t0 = wait_now();
    for (long long i = 0; i < kLimit; i++) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (abort_flag && *abort_flag) return false;
        if (wait_expired(i, t0)) break;
    }
    if (abort_flag) *abort_flag = 1;
    return false;
}
__device__ __forceinline__ void tma_snap(float* dst, const CUtensorMap* map, int x, int y, int z,
                                         uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(tc::smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(tc::smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool test_bar(uint64_t* b, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(tc::smem_u32(b)), "r"(parity)
        : "memory");
    return done != 0;
}

// byte offset of (row o, k) in a 16 x 16 K-major operand (LBO 128, SBO 256)
__device__ __forceinline__ int b_off(int o, int k) {
    return (o >> 3) * 256 + (k >> 3) * 128 + (o & 7) * 16 + (k & 7) * 2;
}
// shared-memory row slot of h1 tile column ix (even positions first)
__device__ __forceinline__ int x_slot(int ix) { return (ix & 1) ? 9 + (ix >> 1) : (ix >> 1); }

// the 9 taps of one kz (K = 32 channels each, two K = 16 MMAs) from the h1
// plane described by dA into the accumulator at column acc, in the tap order
// of the GEMM-engine encoder; the descriptors' start-address field is
// address >> 4 and no operand crosses 256 KB, so offsets add to the field
__device__ __forceinline__ void issue_taps(uint32_t acc, uint64_t dA, uint64_t dB, int kz,
                                           bool first, uint32_t idesc) {
#pragma unroll
    for (int t9 = 0; t9 < 9; t9++) {
        const int ky = t9 / 3, kx = t9 % 3, tap = kz * 9 + t9;
        const int slot0 = kx == 0 ? 0 : (kx == 1 ? 9 : 1);
        const uint32_t off = (uint32_t)(ky * kRowBytes + slot0 * 16);
#pragma unroll
        for (int hh = 0; hh < 2; hh++)
            tc::mma_bf16(acc, dA + (uint64_t)((off + hh * 2 * kKcBytes) >> 4),
                         dB + (uint64_t)((tap * 2 + hh) * 32), idesc,
                         (first && t9 == 0 && hh == 0) ? 0u : 1u);
    }
}

// cursor over the h1 planes of this CTA's items, in order
struct PlaneCursor {
    int item, k, n;  // item index, plane within the item (0 .. 2n), latent planes of the item
    __device__ void start(const Sched& S, int lnz) {
        item = blockIdx.x;
        k = 0;
        n = 0;
        if (item < S.nitems) {
            int cx, cy, z0;
            item_coords(S, lnz, item, cx, cy, z0, n);
        }
    }
    __device__ void next(const Sched& S, int lnz) {
        if (++k == 2 * n + 1) {
            k = 0;
            item += gridDim.x;
            if (item < S.nitems) {
                int cx, cy, z0;
                item_coords(S, lnz, item, cx, cy, z0, n);
            }
        }
    }
    __device__ bool valid(const Sched& S) const { return item < S.nitems; }
};

__global__ void __launch_bounds__(kThreads, 1)
    k_encode_march(const __grid_constant__ EncArgs A, const __grid_constant__ CUtensorMap map,
                   const Sched S, int* status) {
    extern __shared__ uint8_t esm_raw[];
    __shared__ __align__(8) uint64_t snap_full[kSS], snap_free[kSS], h1_full[kSH], h1_free[kSH],
        acc_full[2], acc_free[2], e1a_full[2], e1_done[2], fin;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;

    uint8_t* base = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(esm_raw) + 127) & ~static_cast<uintptr_t>(127));
    uint8_t* w2 = base;
    uint8_t* w1 = base + kW2Bytes;
    float* snap = reinterpret_cast<float*>(w1 + kW1Bytes);
    uint8_t* h1 = w1 + kW1Bytes + kSS * kSnapBytes;
    uint8_t* atile = h1 + kSH * kH1Bytes;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int lnx = A.l.nx, lny = A.l.ny, lnz = A.l.nz;
    volatile int* abrt = &abort_flag;

    if (tid == 0) {
        for (int s = 0; s < kSS; s++) {
            tc::mbar_init(&snap_full[s], 1);
            tc::mbar_init(&snap_free[s], 128);
        }
        for (int s = 0; s < kSH; s++) {
            tc::mbar_init(&h1_full[s], 128);
            tc::mbar_init(&h1_free[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            tc::mbar_init(&acc_full[b], 1);
            tc::mbar_init(&acc_free[b], 128);
            tc::mbar_init(&e1a_full[b], 128);
            tc::mbar_init(&e1_done[b], 1);
        }
        tc::mbar_init(&fin, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tc::tmem_alloc(&tmem_slot, kTmemCols);
    // E2 B operands: (tap, half) -> W2[o][tap][16 half + i], 16 x 16 K-major
    for (int idx = tid; idx < 54 * 16 * 2; idx += kThreads) {
        const int j = idx & 1, o = (idx >> 1) & 15, t = idx >> 5, tap = t >> 1, hh = t & 1;
        float w[8];
#pragma unroll
        for (int e = 0; e < 8; e++) w[e] = A.P[kOW2 + o * 864 + tap * 32 + 16 * hh + 8 * j + e];
        *reinterpret_cast<uint4*>(w2 + t * 512 + b_off(o, 8 * j)) = tc::pack8(w);
    }
    // E1 B operand: W1[o][dz][dy][dx] as k = 0..7 of row o; k = 8..15 zero
    if (tid < 64) {
        const int o = tid >> 1, j = tid & 1;
        float w[8];
#pragma unroll
        for (int e = 0; e < 8; e++) w[e] = j ? 0.f : A.P[kOW1 + o * 8 + e];
        *reinterpret_cast<uint4*>(w1 + (o >> 3) * 256 + j * 128 + (o & 7) * 16) = tc::pack8(w);
    }
    // E1 A tiles: rows past the 561 voxels stay zero (the second K half of
    // row r is row r + 8, multiplied by the zero half of W1, and must be finite)
    for (int i = tid; i < 2 * (kARows - NVOX); i += kThreads) {
        const int g = i / (kARows - NVOX), r = NVOX + i % (kARows - NVOX);
        *reinterpret_cast<uint4*>(atile + g * kATileBytes + r * 16) = make_uint4(0u, 0u, 0u, 0u);
    }
    tc::fence_proxy_async();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- producer: snapshot loads and E2 MMAs ----------------
            // An event loop of non-blocking barrier tests: a snapshot load is
            // issued when its slot is free (at most kLook planes ahead of the MMAs),
            // and the MMAs of h1 plane mp when that plane is complete. Plane 2m of
            // an item closes latent plane m - 1 (kz = 2) and opens latent plane m
            // (kz = 0); plane 2m + 1 is kz = 1 of latent plane m.
            constexpr uint32_t idesc = tc::idesc_bf16(128, 16);
            const uint32_t h1_a = tc::smem_u32(h1);
            const uint64_t dB0 = tc::sdesc(tc::smem_u32(w2), 128, 256);
            int np = 0;  // h1 planes of this CTA
            for (int item = blockIdx.x; item < S.nitems; item += gridDim.x) {
                int cx, cy, z0, nz;
                item_coords(S, lnz, item, cx, cy, z0, nz);
                np += 2 * nz + 1;
            }
            PlaneCursor L, M;
            L.start(S, lnz);
            M.start(S, lnz);
            int l_seq = 0, mp = 0, obase = 0;
            int e1_next[2] = {0, 1};  // next h1 plane of each E1 warpgroup
            constexpr uint32_t idesc1 = tc::idesc_bf16(128, 32);
            const uint64_t dW1 = tc::sdesc(tc::smem_u32(w1), 128, 256);
            long long idle = 0;
            bool ok = true;
            while (mp < np && ok) {
                bool prog = false;
#pragma unroll
                for (int g = 0; g < 2; g++) {
                    const int j = e1_next[g];
                    if (j < np && test_bar(&e1a_full[g], (uint32_t)((j >> 1) & 1))) {
                        // E1 of plane j: 5 M tiles of 128 voxels, K = 16 (8 inputs + 8 zeros)
                        tc::tc_fence_after();
                        const uint32_t a0 = tc::smem_u32(atile + g * kATileBytes);
#pragma unroll
                        for (int t = 0; t < 5; t++)
                            tc::mma_bf16(tmem + kE1Col + g * 160 + t * 32,
                                         tc::sdesc(a0 + t * 2048, 128, 128), dW1, idesc1, 0u);
                        tc::mma_commit(&e1_done[g]);
                        e1_next[g] = j + 2;
                        prog = true;
                    }
                }
                if (l_seq < np && l_seq <= mp + kLook) {
                    const int slot = l_seq % kSS;
                    if (l_seq < kSS || test_bar(&snap_free[slot], (uint32_t)((l_seq / kSS - 1) & 1))) {
                        int lcx, lcy, lz0, lnzi;
                        item_coords(S, lnz, L.item, lcx, lcy, lz0, lnzi);
                        bar_expect(&snap_full[slot], kSnapBytes);
                        tma_snap(snap + slot * (kSnapBytes / 4), &map, 32 * lcx - 4, 64 * lcy - 2,
                                 2 * (2 * lz0 - 1 + L.k), &snap_full[slot]);
                        l_seq++;
                        L.next(S, lnz);
                        prog = true;
                    }
                }
                if (test_bar(&h1_full[mp % kSH], (uint32_t)((mp / kSH) & 1))) {
                    const int k = M.k, n = M.n, m = k >> 1;
                    const bool opens = !(k & 1) && m < n;
                    const int og = obase + m;  // global latent plane opened (k even) or continued
                    if (!opens || og < 2 ||
                        test_bar(&acc_free[og & 1], (uint32_t)(((og >> 1) - 1) & 1))) {
                        tc::tc_fence_after();
                        uint64_t dB;
                        asm volatile("mov.b64 %0, %1;" : "=l"(dB) : "l"(dB0));
                        const uint64_t dA = tc::sdesc(h1_a + (mp % kSH) * kH1Bytes, kKcBytes,
                                                      2 * kRowBytes);
                        if (k & 1) {
                            issue_taps(tmem + (og & 1) * 16, dA, dB, 1, false, idesc);
                        } else {
                            if (m >= 1) {
                                issue_taps(tmem + ((og - 1) & 1) * 16, dA, dB, 2, false, idesc);
                                tc::mma_commit(&acc_full[(og - 1) & 1]);
                            }
                            if (opens) issue_taps(tmem + (og & 1) * 16, dA, dB, 0, true, idesc);
                        }
                        tc::mma_commit(&h1_free[mp % kSH]);
                        mp++;
                        if (M.k + 1 == 2 * M.n + 1) obase += M.n;
                        M.next(S, lnz);
                        prog = true;
                    }
                }
                if (prog) {
                    idle = 0;
                } else if (++idle > kIdleLimit || *abrt) {
                    ok = false;
                }
            }
            if (!ok) {
                *abrt = 1;
                // copies still in flight must land before the CTA leaves: wait
                // (bounded, ignoring the flag) for every snapshot slot's last load
                for (int s = (l_seq > kSS ? l_seq - kSS : 0); s < l_seq; s++)
                    wait_bar(&snap_full[s % kSS], (uint32_t)((s / kSS) & 1), nullptr);
            }
            tc::mma_commit(&fin);
            if (!wait_bar(&fin, 0, nullptr)) *abrt = 1;
        }
    } else if (warp <= 8) {
        // ---------------- E1: two warpgroups, alternate h1 planes ----------------
        // per plane: A tile rows = bf16(s / rms) of each h1 voxel's 2 x 2 x 2 patch;
        // the producer's MMAs put W1 x0 into this warpgroup's TMEM columns; the
        // epilogue adds b1, applies LeakyReLU, rounds to bf16 and stores h1
        const int g = (warp - 1) >> 2, t = tid - 32 - 128 * g, q = warp & 3;
        uint8_t* at = atile + g * kATileBytes;
        const uint32_t tcol = tmem + kE1Col + g * 160 + ((uint32_t)(q * 32) << 16);
        float b1[32];
#pragma unroll
        for (int c = 0; c < 32; c++) b1[c] = A.P[kOB1 + c];
        const float inv_s = *A.inv_sigma;
        PlaneCursor C;
        C.start(S, lnz);
        bool ok = true;
        for (int j = 0; C.valid(S) && ok; j++, C.next(S, lnz)) {
            if ((j & 1) != g) continue;
            int cx, cy, z0, nz;
            item_coords(S, lnz, C.item, cx, cy, z0, nz);
            const int hz = 2 * z0 - 1 + C.k;
            ok = wait_bar(&snap_full[j % kSS], (uint32_t)((j / kSS) & 1), abrt);
            if (!ok) break;
            const float* sp = snap + (j % kSS) * (kSnapBytes / 4);
            for (int v = t; v < NVOX; v += 128) {
                const int iy = v / HX, ix = v - iy * HX;
                float x[8];
#pragma unroll
                for (int dz = 0; dz < 2; dz++)
#pragma unroll
                    for (int dy = 0; dy < 2; dy++) {
                        const float2 p2 = *reinterpret_cast<const float2*>(
                            sp + (dz * SYR + 2 * iy + dy) * SX + 2 + 2 * ix);
                        x[dz * 4 + dy * 2] = p2.x * inv_s;
                        x[dz * 4 + dy * 2 + 1] = p2.y * inv_s;
                    }
                *reinterpret_cast<uint4*>(at + v * 16) = tc::pack8(x);
            }
            tc::fence_proxy_async();
            bar_arrive(&snap_free[j % kSS]);
            bar_arrive(&e1a_full[g]);
            ok = wait_bar(&e1_done[g], (uint32_t)((j >> 1) & 1), abrt);
            if (ok && j >= kSH) ok = wait_bar(&h1_free[j % kSH], (uint32_t)((j / kSH - 1) & 1), abrt);
            if (!ok) break;
            tc::tc_fence_after();
            uint8_t* hp = h1 + (j % kSH) * kH1Bytes;
            const bool zin = hz >= 0 && hz < A.h.nz;
#pragma unroll 1
            for (int mt = 0; mt < 5; mt++) {
                const int v0 = mt * 128 + q * 32;
                if (v0 >= NVOX) break;  // warp-uniform
                float acc[32];
                tc::tmem_ld16(tcol + mt * 32, acc);
                tc::tmem_ld16(tcol + mt * 32 + 16, acc + 16);
                const int v = v0 + lane;
                if (v < NVOX) {
                    const int iy = v / HX, ix = v - iy * HX;
                    const int hy = 32 * cy - 1 + iy, hx = 16 * cx - 1 + ix;
                    const bool in = zin && hy >= 0 && hy < A.h.ny && hx >= 0 && hx < A.h.nx;
                    uint8_t* dst = hp + iy * kRowBytes + x_slot(ix) * 16;
#pragma unroll
                    for (int kc = 0; kc < 4; kc++) {
                        float hv[8];
#pragma unroll
                        for (int c = 0; c < 8; c++) hv[c] = lrelu(acc[8 * kc + c] + b1[8 * kc + c]);
                        *reinterpret_cast<uint4*>(dst + kc * kKcBytes) =
                            in ? tc::pack8(hv) : make_uint4(0u, 0u, 0u, 0u);
                    }
                }
            }
            tc::tc_fence_before();
            tc::fence_proxy_async();
            bar_arrive(&h1_full[j % kSH]);
        }
    } else {
        // ---------------- latent epilogue: warpgroup 3 ----------------
        const int row = tid & 127, ly = row >> 3, lx = row & 7;
        const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
        float b2[16];
#pragma unroll
        for (int o = 0; o < 16; o++) b2[o] = A.P[kOB2 + o];
        int out = 0;
        bool ok = true;
        for (int item = blockIdx.x; item < S.nitems && ok; item += gridDim.x) {
            int cx, cy, z0, nz;
            item_coords(S, lnz, item, cx, cy, z0, nz);
            const int X = cx * TX + lx, Y = cy * TY + ly;
            for (int zi = 0; zi < nz; zi++, out++) {
                const int b = out & 1, u = out >> 1;
                ok = wait_bar(&acc_full[b], (uint32_t)(u & 1), abrt);
                if (!ok) break;
                tc::tc_fence_after();
                float acc[16];
                tc::tmem_ld16(lane_base + b * 16, acc);
                tc::tc_fence_before();
                bar_arrive(&acc_free[b]);
                if (X < lnx && Y < lny) {
#pragma unroll
                    for (int o = 0; o < 16; o++) acc[o] += b2[o];
                    uint4* dst = reinterpret_cast<uint4*>(
                        A.lat + ((((long long)(z0 + zi) * lny + Y) * lnx + X) * 16));
                    dst[0] = tc::pack8(acc);
                    dst[1] = tc::pack8(acc + 8);
                }
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (tid == 0 && *abrt && status) atomicCAS(status, 0, tc::kErrTimeout);
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, kTmemCols);
    }
}

// 0 automatic (z-marching kernel when TMA is available), 1 GEMM-engine
// encoder, 2 z-marching kernel
int g_encoder = 0;

}  // namespace
}  // namespace ae

void ae_set_encoder(int which) { ae::g_encoder = which; }

// latent of the snapshot `in` scaled by *inv_sigma; cudaErrorNotSupported when
// the kernel cannot run (no tensor-map encoder, misaligned snapshot rows or
// latent, or not selected): the caller then runs the GEMM-engine encoder
cudaError_t ae_encode_march(const float* P, const ae::Vol& in, const float* inv_sigma,
                            ae::bf16* lat, int* status, cudaStream_t s) {
    using namespace ae;
    if (g_encoder == 1) return cudaErrorNotSupported;
    EncodeTiledFn enc = tma_encoder();
    if (!enc || (reinterpret_cast<uintptr_t>(in.p) & 15) || (in.sy % 4) || (in.sz % 4) ||
        (reinterpret_cast<uintptr_t>(lat) & 15))
        return cudaErrorNotSupported;
    static int nsm = 0;
    if (nsm == 0) {
        cudaError_t e = cudaFuncSetAttribute(k_encode_march,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
        if (e != cudaSuccess) return e;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (nsm < 1) nsm = 1;
    }
    CUtensorMap map;
    memset(&map, 0, sizeof map);
    const cuuint64_t dims[3] = {(cuuint64_t)in.nx, (cuuint64_t)in.ny, (cuuint64_t)in.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)in.sy * 4, (cuuint64_t)in.sz * 4};
    const cuuint32_t box[3] = {SX, SYR, 2};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(in.p), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorNotSupported;
    const Dims3 l{in.nx / 4, in.ny / 4, in.nz / 4}, h{in.nx / 2, in.ny / 2, in.nz / 2};
    Sched S;
    S.ncx = (l.nx + TX - 1) / TX;
    S.ncy = (l.ny + TY - 1) / TY;
    const long long ncol = (long long)S.ncx * S.ncy;
    // z chunk: smallest per-CTA makespan, each chunk's extra h1 plane counted
    // as half a latent plane of work
    long long best = -1;
    S.zc = l.nz;
    for (int zc = std::min(4, l.nz); zc <= l.nz; zc++) {
        const long long items = ncol * ((l.nz + zc - 1) / zc);
        const long long span = (items + nsm - 1) / nsm * (2 * zc + 1);
        if (best < 0 || span < best) {
            best = span;
            S.zc = zc;
        }
    }
    S.nitems = (int)(ncol * ((l.nz + S.zc - 1) / S.zc));
    EncArgs a{P, inv_sigma, lat, l, h};
    const int grid = std::min(nsm, S.nitems);
    k_encode_march<<<grid, kThreads, kSmem, s>>>(a, map, S, status);
    return cudaGetLastError();
}

}  // namespace rtm
