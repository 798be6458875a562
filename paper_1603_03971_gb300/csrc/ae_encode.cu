// Inference encoder, z-marching: E1 (patch conv 1 -> 32, kernel 2, stride 2)
// + LeakyReLU + E2 (conv 32 -> 16, kernel 3, stride 2, padding 1) in one
// persistent kernel, one CTA per SM. The 32-channel intermediate h1 never
// leaves shared memory.
//
// Work item: a column of 8 x 16 latent voxels (x, y) over a range of latent
// planes z. Latent plane z reads h1 planes 2z - 1, 2z, 2z + 1; each h1 plane
// of the column is a 17 x 33 tile (one h1 voxel of halo on the low side)
// computed from two snapshot planes, which TMA copies (40 x 66 floats, zeros
// outside the volume) into a three-slot ring; a loader thread (warp 13)
// issues each copy as soon as its slot is free.
//
// E1 runs on the tensor cores as well. Two E1 roles of 128 threads (warps
// 1-4: even h1 planes, warps 5-8: odd ones) each write, for their plane,
// the bf16(s / rms) values of every h1 voxel's 2 x 2 x 2 patch as one row of
// a 648-row A tile (rows in h1 slot order, below: row 17 iy + slot, so that
// one float4 of the snapshot row serves two voxels and the epilogue's
// stores are contiguous); once all 128 threads have written their rows
// (mbarrier of 128 arrivals) the role's first thread issues 5 tcgen05.mma (M = 128 voxels,
// N = 32, K = 16: the 8 patch values, then 8 columns multiplied by the zero
// half of W1) into the role's 160 TMEM columns. Each warp of a role reads
// the 32 channels of its 32 TMEM lanes, one M tile loading while the one
// before it is processed, adds b1, applies LeakyReLU (packed f32x2 arithmetic),
// rounds to bf16 and stores h1 into a three-slot ring laid out as E2's A
// operand in the canonical K-major no-swizzle layout: four 8-channel
// core-matrix columns (leading byte offset 8976 B) of [33][17] 16-byte
// rows, with the x positions split by parity (9 even, then 8 odd) so that
// every tap of the stride-2 convolution reads 8 consecutive rows: tap (kz,
// ky, kx) of latent row (ly, lx) is h1 row 2 ly + ky, slot lx (kx = 0), 9 +
// lx (kx = 1) or lx + 1 (kx = 2); 8-row groups (one per ly) are 544 B apart.
// The products, sums and rounding points are those of the GEMM-engine
// encoder, so the latents are the same.
//
// E2 runs on the tensor cores, one h1 plane at a time: as soon as plane p is
// complete, the E2 issuer (warp 0) issues its 9 taps x 2 K halves of
// tcgen05.mma (M = 128 latent voxels, K = 16 channels) into the accumulator
// of every latent plane that reads it (plane 2m: kz = 2 of latent m - 1 and
// kz = 0 of latent m, as N = 32 MMAs into both accumulators at once after a
// first tap of two N = 16 MMAs; plane 2m + 1: kz = 1 of latent m, N = 16),
// so each latent sums its 27 taps in the order of the GEMM-engine encoder
// and each h1 slot is freed after one use. Two 16-column accumulators
// (TMEM columns 0-15 and 16-31) alternate between latent planes; warps
// 9-12 add b2, round to bf16 and store the latent rows. mbarriers:
// snapshot full (TMA bytes) / free (128 arrivals), A tile full (128
// arrivals) / E1 done (commit), h1 full (128 arrivals) / free (commit),
// accumulator full (commit) / free (128 arrivals). Every wait is bounded,
// shares an abort flag and sleeps in the mbarrier poll instead of spinning.
//
// Measured with per-stage clock stamps at 384^3 (one h1 plane every ~2600
// cycles per CTA): a single issuing thread for E1 and E2, snapshot copies
// and E2 MMAs in one event loop made the E1 MMAs wait ~1900 cycles per plane
// behind the E2 issue, and the epilogue of one plane took ~4000 cycles with
// unpipelined TMEM loads and scalar arithmetic; pairing the kz = 2 and
// kz = 0 MMAs cut the E2 issue from ~2060 to ~1560 cycles per plane. With
// the epilogue pipelined and packed, roles of one warpgroup (14 warps per
// SM) run 2 % faster than roles of two warpgroups (22 warps) that split the
// channels.

#include <cuda.h>
#include <cuda_bf16.h>
#include <string.h>

#include <algorithm>

#include "../../include/rtm.h"
#include "ae_internal.h"
#include "packed_f32x2.cuh"
#include "rtm_internal.h"
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
static_assert(32 * kRowBytes + 16 * 16 < 65536, "h1 row offsets fit 16 bits");
constexpr int SX = 40, SYR = 2 * HY;                     // snapshot box: 40 x 66 x 2
constexpr int kSnapBytes = SX * SYR * 2 * 4;             // 21120
// E2 B operands, per (tap t9 of a kz, K half): region C holds kz = 2 and 0
// as a 48-row block [kz 2 | kz 0 | kz 2] (1536 B), so that 16-row operands of
// either kz and 32-row operands of both, in either order, are contiguous;
// region K1 holds kz = 1 (16 rows, 512 B)
constexpr int kW2CBlock = 1536, kW2CBytes = 18 * kW2CBlock;
constexpr int kW2Bytes = kW2CBytes + 18 * 512;
constexpr int kSS = 3, kSH = 3;
constexpr int kW1Bytes = 1024;      // W1 as a 32 x 16 operand (k 8..15 zero)
constexpr int kARows = 648;         // E1 A tile: 5 M tiles of 128 rows + 8 rows read as K half 2
constexpr int kATileBytes = kARows * 16;                 // 10368
constexpr int kE1Col = 32;          // E1 accumulators: 2 x (5 x 32) TMEM columns from here
constexpr int kSmem = 128 + kW2Bytes + kW1Bytes + kSS * kSnapBytes + kSH * kH1Bytes +
                      2 * kATileBytes;
static_assert(kSmem + 1024 <= 227 * 1024, "shared memory of one CTA");
constexpr int kE1Threads = 128;  // threads of one E1 role (one warpgroup)
constexpr int kThreads = 14 * 32;
constexpr int kTmemCols = 512;
constexpr long long kLimit = 1LL << 24;
constexpr uint32_t kSuspendNs = 20000;  // longest sleep of one poll (woken by the phase)

struct Sched {
    int ncx, ncy, zc, nitems;
};

struct EncArgs {
    const float* P;
    const float* inv_sigma;
    bf16* lat;
    Dims3 l, h;
    int stall;  // >= 0: CTA 0's copy of the h1 plane that many before its last
                // expects 16 bytes too many (test)
};

__device__ __forceinline__ void item_coords(const Sched& S, int lnz, int item, int& cx, int& cy,
                                            int& z0, int& nz) {
    cx = item % S.ncx;
    cy = (item / S.ncx) % S.ncy;
    z0 = (item / (S.ncx * S.ncy)) * S.zc;
    nz = min(S.zc, lnz - z0);
}

static_assert(kSlope > 0.f && kSlope < 1.f, "LeakyReLU as a maximum needs 0 < slope < 1");

__device__ __forceinline__ void bar_expect(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(b)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(b)) : "memory");
}
// bounded wait (2 s of %globaltimer, the poll count as a backstop); gives up
// early once another thread has raised the abort flag, where one is given.
// Each poll may sleep until the phase completes
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
__device__ __forceinline__ void tma_snap(float* dst, const CUtensorMap* map, int x, int y, int z,
                                         uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(tc::smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(tc::smem_u32(bar))
        : "memory");
}

// 16 columns at a TMEM address (one M tile) of this warp's lanes into r,
// without waiting: the registers must not be read before tmem_wait_regs(r)
__device__ __forceinline__ void tmem_ld16_nw(uint32_t a0, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(a0)
        : "memory");
}
// wait for this thread's TMEM loads; the registers are operands, so no read
// of them can be scheduled before the wait
__device__ __forceinline__ void tmem_wait_regs(uint32_t* r) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                   "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                   "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
                 :
                 : "memory");
}

// byte offset of (row o, k) in a 16 x 16 K-major operand (LBO 128, SBO 256)
__device__ __forceinline__ int b_off(int o, int k) {
    return (o >> 3) * 256 + (k >> 3) * 128 + (o & 7) * 16 + (k & 7) * 2;
}

// byte offset of the h1 rows that tap t9 (ky, kx) of a latent row reads
__device__ __forceinline__ uint32_t tap_off(int t9) {
    const int ky = t9 / 3, kx = t9 % 3;
    const int slot0 = kx == 0 ? 0 : (kx == 1 ? 9 : 1);
    return (uint32_t)(ky * kRowBytes + slot0 * 16);
}

// the 9 taps of one kz (K = 32 channels each, two K = 16 MMAs, N = 16) from
// the h1 plane described by dA into the accumulator at column acc, in the tap
// order of the GEMM-engine encoder; dB addresses the kz's operand of tap 0,
// K half 0, and (t9, half) operands are `stride` bytes apart. The
// descriptors' start-address field is address >> 4 and no operand crosses
// 256 KB, so offsets add to the field
__device__ __forceinline__ void issue_taps(uint32_t acc, uint64_t dA, uint64_t dB, int stride,
                                           bool first, uint32_t idesc) {
#pragma unroll
    for (int t9 = 0; t9 < 9; t9++) {
        const uint32_t off = tap_off(t9);
#pragma unroll
        for (int hh = 0; hh < 2; hh++)
            tc::mma_bf16(acc, dA + (uint64_t)((off + hh * 2 * kKcBytes) >> 4),
                         dB + (uint64_t)(((t9 * 2 + hh) * stride) >> 4), idesc,
                         (first && t9 == 0 && hh == 0) ? 0u : 1u);
    }
}

// an h1 plane that closes one latent plane (kz = 2, accumulating) and opens
// the next (kz = 0): the first tap as two N = 16 MMAs (the opening
// accumulator is overwritten), the other 17 as N = 32 MMAs into both
// accumulators at once (columns 0-31; B rows 0-15 go to columns 0-15).
// kz0_low: the opening plane's accumulator is columns 0-15
__device__ __forceinline__ void issue_pair(uint32_t tmem, uint64_t dA, uint64_t dC, bool kz0_low,
                                           uint32_t idesc16, uint32_t idesc32) {
    const uint32_t acc_open = tmem + (kz0_low ? 0 : 16), acc_close = tmem + (kz0_low ? 16 : 0);
    const uint64_t dB32 = dC + (uint64_t)((kz0_low ? 512 : 0) >> 4);
    const uint32_t off0 = tap_off(0);
    tc::mma_bf16(acc_close, dA + (uint64_t)(off0 >> 4), dC, idesc16, 1u);
    tc::mma_bf16(acc_open, dA + (uint64_t)(off0 >> 4), dC + (uint64_t)(512 >> 4), idesc16, 0u);
#pragma unroll
    for (int t9 = 0; t9 < 9; t9++) {
        const uint32_t off = tap_off(t9);
#pragma unroll
        for (int hh = 0; hh < 2; hh++) {
            if (t9 == 0 && hh == 0) continue;
            tc::mma_bf16(tmem, dA + (uint64_t)((off + hh * 2 * kKcBytes) >> 4),
                         dB32 + (uint64_t)(((t9 * 2 + hh) * kW2CBlock) >> 4), idesc32, 1u);
        }
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
            tc::mbar_init(&snap_free[s], kE1Threads);
        }
        for (int s = 0; s < kSH; s++) {
            tc::mbar_init(&h1_full[s], kE1Threads);
            tc::mbar_init(&h1_free[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            tc::mbar_init(&acc_full[b], 1);
            tc::mbar_init(&acc_free[b], 128);
            tc::mbar_init(&e1a_full[b], kE1Threads);
            tc::mbar_init(&e1_done[b], 1);
        }
        tc::mbar_init(&fin, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tc::tmem_alloc(&tmem_slot, kTmemCols);
    // E2 B operands: (tap, half) -> W2[o][tap][16 half + i], 16-row K-major
    // blocks in region C (kz 0 and 2) or K1 (kz 1)
    for (int idx = tid; idx < 54 * 16 * 2; idx += kThreads) {
        const int j = idx & 1, o = (idx >> 1) & 15, t = idx >> 5, tap = t >> 1, hh = t & 1;
        float w[8];
#pragma unroll
        for (int e = 0; e < 8; e++) w[e] = A.P[kOW2 + o * 864 + tap * 32 + 16 * hh + 8 * j + e];
        const uint4 v = tc::pack8(w);
        const int kz = tap / 9, blk = (tap % 9) * 2 + hh, bo = b_off(o, 8 * j);
        if (kz == 1) {
            *reinterpret_cast<uint4*>(w2 + kW2CBytes + blk * 512 + bo) = v;
        } else if (kz == 0) {
            *reinterpret_cast<uint4*>(w2 + blk * kW2CBlock + 512 + bo) = v;
        } else {
            *reinterpret_cast<uint4*>(w2 + blk * kW2CBlock + bo) = v;
            *reinterpret_cast<uint4*>(w2 + blk * kW2CBlock + 1024 + bo) = v;
        }
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
            // ---------------- E2 issuer ----------------
            // the MMAs of h1 plane mp once that plane is complete (and, for a
            // plane that opens a latent plane, once its accumulator is free).
            // Plane 2m of an item closes latent plane m - 1 (kz = 2) and opens
            // latent plane m (kz = 0); plane 2m + 1 is kz = 1 of latent plane m.
            constexpr uint32_t idesc = tc::idesc_bf16(128, 16), idesc32 = tc::idesc_bf16(128, 32);
            const uint32_t h1_a = tc::smem_u32(h1);
            const uint64_t dB0 = tc::sdesc(tc::smem_u32(w2), 128, 256);
            PlaneCursor M;
            M.start(S, lnz);
            int obase = 0;
            bool ok = true;
            for (int mp = 0; M.valid(S); mp++) {
                ok = wait_bar(&h1_full[mp % kSH], (uint32_t)((mp / kSH) & 1), abrt);
                if (!ok) break;
                const int k = M.k, n = M.n, m = k >> 1;
                const bool opens = !(k & 1) && m < n;
                const int og = obase + m;  // global latent plane opened (k even) or continued
                if (opens && og >= 2)
                    ok = wait_bar(&acc_free[og & 1], (uint32_t)(((og >> 1) - 1) & 1), abrt);
                if (!ok) break;
                tc::tc_fence_after();
                uint64_t dB;
                asm volatile("mov.b64 %0, %1;" : "=l"(dB) : "l"(dB0));
                const uint64_t dA =
                    tc::sdesc(h1_a + (mp % kSH) * kH1Bytes, kKcBytes, 2 * kRowBytes);
                // dB: region C (kz 2 at +0, kz 0 at +512); region K1 at +kW2CBytes
                if (k & 1) {
                    issue_taps(tmem + (og & 1) * 16, dA, dB + (uint64_t)(kW2CBytes >> 4), 512,
                               false, idesc);
                } else if (m >= 1 && opens) {
                    issue_pair(tmem, dA, dB, (og & 1) == 0, idesc, idesc32);
                    tc::mma_commit(&acc_full[(og - 1) & 1]);
                } else if (m >= 1) {
                    issue_taps(tmem + ((og - 1) & 1) * 16, dA, dB, kW2CBlock, false, idesc);
                    tc::mma_commit(&acc_full[(og - 1) & 1]);
                } else if (opens) {
                    issue_taps(tmem + (og & 1) * 16, dA, dB + (uint64_t)(512 >> 4), kW2CBlock,
                               true, idesc);
                }
                tc::mma_commit(&h1_free[mp % kSH]);
                if (M.k + 1 == 2 * M.n + 1) obase += M.n;
                M.next(S, lnz);
            }
            if (!ok) *abrt = 1;
            tc::mma_commit(&fin);
            if (!wait_bar(&fin, 0, nullptr)) *abrt = 1;
        }
    } else if (warp <= 8) {
        // ---------------- E1: two roles of 4 warps, alternate h1 planes ----------------
        // per plane: A tile rows = bf16(s / rms) of each h1 voxel's 2 x 2 x 2 patch;
        // the role's first thread puts W1 x0 into the role's TMEM columns; the
        // epilogue adds b1, applies LeakyReLU, rounds to bf16 and stores h1.
        // Role g = warps 1 + 4 g .. 4 + 4 g; a warp reads TMEM lanes 32 (warp % 4)
        // .. + 31, all 32 h1 channels
        const int g = (warp - 1) >> 2, t = tid - 32 - kE1Threads * g, q = warp & 3;
        uint8_t* at = atile + g * kATileBytes;
        const uint32_t tcol = tmem + kE1Col + g * 160 + ((uint32_t)(q * 32) << 16);
        constexpr uint32_t idesc1 = tc::idesc_bf16(128, 32);
        const uint64_t dW1 = tc::sdesc(tc::smem_u32(w1), 128, 256);
        // b1 as pairs, and the slope as a pair:
        // packed f32x2 adds and multiplies (IEEE single precision per lane)
        uint64_t b1p[16];
#pragma unroll
        for (int c = 0; c < 16; c++)
            b1p[c] = f32x2::pack(A.P[kOB1 + 2 * c], A.P[kOB1 + 2 * c + 1]);
        const uint64_t slope2 = f32x2::pack(kSlope, kSlope);
        const float inv_s = *A.inv_sigma;
        // per item: this thread's h1 row offset in each M tile (16 bits each,
        // two per word: every offset is below 2^15) and whether the row's
        // voxel lies inside the h1 volume in x and y (bit mt)
        uint32_t tile_off[3];
        uint32_t in_xy = 0;
        int cur_item = -1;
        PlaneCursor C;
        C.start(S, lnz);
        bool ok = true;
        for (int j = 0; C.valid(S) && ok; j++, C.next(S, lnz)) {
            if ((j & 1) != g) continue;
            int cx, cy, z0, nz;
            item_coords(S, lnz, C.item, cx, cy, z0, nz);
            if (C.item != cur_item) {
                cur_item = C.item;
                in_xy = 0;
                tile_off[0] = tile_off[1] = tile_off[2] = 0;
#pragma unroll
                for (int mt = 0; mt < 5; mt++) {
                    const int r = mt * 128 + q * 32 + lane;
                    const int iy = r / HX, sl = r - iy * HX;
                    const int ix = sl < 9 ? 2 * sl : 2 * sl - 17;
                    const int hy = 32 * cy - 1 + iy, hx = 16 * cx - 1 + ix;
                    tile_off[mt >> 1] |= (uint32_t)(iy * kRowBytes + sl * 16) << (16 * (mt & 1));
                    if (r < NVOX && hy >= 0 && hy < A.h.ny && hx >= 0 && hx < A.h.nx)
                        in_xy |= 1u << mt;
                }
            }
            const int hz = 2 * z0 - 1 + C.k;
            // the slot's previous plane (the other role's) released first: then
            // its copy has landed, and this wait's parity names this plane's
            // phase and not that earlier, still incomplete one
            ok = j < kSS || wait_bar(&snap_free[j % kSS], (uint32_t)((j / kSS - 1) & 1), abrt);
            if (ok) ok = wait_bar(&snap_full[j % kSS], (uint32_t)((j / kSS) & 1), abrt);
            if (!ok) break;
            const float* sp = snap + (j % kSS) * (kSnapBytes / 4);
            // A tile rows in h1 slot order: row 17 iy + slot. Unit (iy, p) reads
            // the snapshot float4 at box x = 4 p, which holds the patch columns
            // of h1 x positions 2 p - 1 (slot 8 + p; none for p = 0) and 2 p
            // (slot p)
            for (int u = t; u < HY * 9; u += kE1Threads) {
                const int iy = u / 9, p = u - iy * 9;
                float xe[8], xo[8];
#pragma unroll
                for (int dz = 0; dz < 2; dz++)
#pragma unroll
                    for (int dy = 0; dy < 2; dy++) {
                        const float4 p4 = *reinterpret_cast<const float4*>(
                            sp + (dz * SYR + 2 * iy + dy) * SX + 4 * p);
                        xo[dz * 4 + dy * 2] = p4.x * inv_s;
                        xo[dz * 4 + dy * 2 + 1] = p4.y * inv_s;
                        xe[dz * 4 + dy * 2] = p4.z * inv_s;
                        xe[dz * 4 + dy * 2 + 1] = p4.w * inv_s;
                    }
                *reinterpret_cast<uint4*>(at + (iy * HX + p) * 16) = tc::pack8(xe);
                if (p > 0) *reinterpret_cast<uint4*>(at + (iy * HX + 8 + p) * 16) = tc::pack8(xo);
            }
            tc::fence_proxy_async();
            bar_arrive(&snap_free[j % kSS]);
            bar_arrive(&e1a_full[g]);
            bool issued = false;
            if (t == 0) {
                // E1 of plane j once all 128 rows are written: 5 M tiles of
                // 128 voxels, K = 16 (8 inputs + 8 zeros)
                ok = wait_bar(&e1a_full[g], (uint32_t)((j >> 1) & 1), abrt);
                if (ok) {
                    issued = true;
                    tc::tc_fence_after();
                    const uint32_t a0 = tc::smem_u32(at);
#pragma unroll
                    for (int mt = 0; mt < 5; mt++)
                        tc::mma_bf16(tmem + kE1Col + g * 160 + mt * 32,
                                     tc::sdesc(a0 + mt * 2048, 128, 128), dW1, idesc1, 0u);
                    tc::mma_commit(&e1_done[g]);
                }
            }
            if (ok) ok = wait_bar(&e1_done[g], (uint32_t)((j >> 1) & 1), abrt);
            // the MMAs must be done with the tile and the accumulator before
            // an aborting CTA frees its tensor memory: wait, ignoring the flag
            if (!ok && issued) wait_bar(&e1_done[g], (uint32_t)((j >> 1) & 1), nullptr);
            if (ok && j >= kSH) ok = wait_bar(&h1_free[j % kSH], (uint32_t)((j / kSH - 1) & 1), abrt);
            if (!ok) break;
            tc::tc_fence_after();
            uint8_t* hp = h1 + (j % kSH) * kH1Bytes;
            const bool zin = hz >= 0 && hz < A.h.nz;
            // one M tile's 32 channels: b1, LeakyReLU as max(h, slope h) (the
            // same bits as the select form for 0 < slope < 1), bf16, four
            // 16-byte stores; consecutive lanes hold consecutive slots, so the
            // stores are conflict-free. Each tile after the first loads while
            // the one before it is stored (a loaded register becomes readable
            // a few hundred cycles after the load is issued); tiles 0-3 hold
            // rows of every warp (row 384 + 127 < 561), tile 4 only those of
            // the warps whose rows start below 561
            auto store_tile = [&](int mt, const uint32_t* acc) {
                if (mt * 128 + q * 32 + lane >= NVOX) return;
                const bool in = zin && ((in_xy >> mt) & 1u);
                uint8_t* dst = hp + ((tile_off[mt >> 1] >> (16 * (mt & 1))) & 0xFFFFu);
#pragma unroll
                for (int kc = 0; kc < 4; kc++) {
                    uint32_t w[4];
#pragma unroll
                    for (int c = 0; c < 4; c++) {
                        const int i = 8 * kc + 2 * c;
                        const uint64_t h = f32x2::add(
                            f32x2::pack(__uint_as_float(acc[i]), __uint_as_float(acc[i + 1])),
                            b1p[i >> 1]);
                        const uint64_t sh = f32x2::mul(h, slope2);
                        float h0, h1, s0, s1;
                        f32x2::unpack(h, h0, h1);
                        f32x2::unpack(sh, s0, s1);
                        w[c] = in ? tc::pack2(fmaxf(h0, s0), fmaxf(h1, s1)) : 0u;
                    }
                    *reinterpret_cast<uint4*>(dst + kc * kKcBytes) = make_uint4(w[0], w[1], w[2], w[3]);
                }
            };
            const bool t4 = 4 * 128 + q * 32 < NVOX;  // warp-uniform
            uint32_t x0[32], x1[32];
            tmem_ld16_nw(tcol, x0);
            tmem_ld16_nw(tcol + 16, x0 + 16);
            tmem_wait_regs(x0);
            tmem_wait_regs(x0 + 16);
            tmem_ld16_nw(tcol + 32, x1);
            tmem_ld16_nw(tcol + 48, x1 + 16);
            store_tile(0, x0);
            tmem_wait_regs(x1);
            tmem_wait_regs(x1 + 16);
            tmem_ld16_nw(tcol + 64, x0);
            tmem_ld16_nw(tcol + 80, x0 + 16);
            store_tile(1, x1);
            tmem_wait_regs(x0);
            tmem_wait_regs(x0 + 16);
            tmem_ld16_nw(tcol + 96, x1);
            tmem_ld16_nw(tcol + 112, x1 + 16);
            store_tile(2, x0);
            tmem_wait_regs(x1);
            tmem_wait_regs(x1 + 16);
            if (t4) {
                tmem_ld16_nw(tcol + 128, x0);
                tmem_ld16_nw(tcol + 144, x0 + 16);
            }
            store_tile(3, x1);
            if (t4) {
                tmem_wait_regs(x0);
                tmem_wait_regs(x0 + 16);
                store_tile(4, x0);
            }
            tc::tc_fence_before();
            tc::fence_proxy_async();
            bar_arrive(&h1_full[j % kSH]);
        }
    } else if (warp <= 12) {
        // ---------------- latent epilogue: warps 9-12 ----------------
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
    } else if (lane == 0) {
        // ---------------- snapshot loader: warp 13 ----------------
        // each h1 plane's two snapshot planes into the next ring slot once
        // the role that used the slot last has built its A tile from it
        int np = 0;  // h1 planes of this CTA
        for (int item = blockIdx.x; item < S.nitems; item += gridDim.x) {
            int cx, cy, z0, nz;
            item_coords(S, lnz, item, cx, cy, z0, nz);
            np += 2 * nz + 1;
        }
        PlaneCursor L;
        L.start(S, lnz);
        int l_seq = 0;
        for (; L.valid(S); l_seq++, L.next(S, lnz)) {
            const int slot = l_seq % kSS;
            if (l_seq >= kSS &&
                !wait_bar(&snap_free[slot], (uint32_t)((l_seq / kSS - 1) & 1), abrt))
                break;
            int lcx, lcy, lz0, lnzi;
            item_coords(S, lnz, L.item, lcx, lcy, lz0, lnzi);
            // a test-armed stall: this copy's phase never completes, so the
            // wait for it runs out (rtm_set_test_stall). It is one of the
            // CTA's last kSS copies: no later copy reuses its slot, so no
            // wait can take a later phase of its mbarrier for the stuck one
            const bool stalled =
                A.stall >= 0 && A.stall < kSS && l_seq == np - 1 - A.stall && blockIdx.x == 0;
            bar_expect(&snap_full[slot], kSnapBytes + (stalled ? 16u : 0u));
            tma_snap(snap + slot * (kSnapBytes / 4), &map, 32 * lcx - 4, 64 * lcy - 2,
                     2 * (2 * lz0 - 1 + L.k), &snap_full[slot]);
        }
        // every copy must land before the CTA leaves (after an abort some were
        // never waited for): wait, bounded and ignoring the flag, for each
        // slot's last load; a completed one answers at once
        for (int q = (l_seq > kSS ? l_seq - kSS : 0); q < l_seq; q++)
            wait_bar(&snap_full[q % kSS], (uint32_t)((q / kSS) & 1), nullptr);
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
    EncArgs a{P, inv_sigma, lat, l, h, take_test_stall(RTM_STALL_ENCODER)};
    const int grid = std::min(nsm, S.nitems);
    k_encode_march<<<grid, kThreads, kSmem, s>>>(a, map, S, status);
    return cudaGetLastError();
}

}  // namespace rtm
