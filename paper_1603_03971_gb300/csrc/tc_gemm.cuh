// Tensor-core (tcgen05) GEMM engine for the snapshot codec.
//
// One 128-thread CTA computes a 128 x N tile of C = A * B (N = 16 or 32),
// bfloat16 operands, float32 accumulation in tensor memory. The operation
// type Op decides how each 128 x 32 slab of A and N x 32 slab of B is
// gathered from global memory (convolution windows, transposes, fused
// normalisation) and what the epilogue does with the accumulator rows.
//
// Shared-memory operand layout: canonical K-major, no swizzle. An 8-row x
// 16-byte core matrix is contiguous; core matrices adjacent in K are 128 B
// apart (leading byte offset), 8-row groups are 512 B apart (stride byte
// offset), so a 32-wide K slab of R rows takes R * 64 bytes.
//
// Pipeline: S shared-memory stages. All threads gather slab i into stage
// i % S (after the MMAs that read slab i - S have completed, signalled on
// that stage's mbarrier by tcgen05.commit), fence the generic-proxy writes
// for the async proxy, synchronise, and one thread issues two K = 16
// tcgen05.mma instructions and a commit. After the last slab the
// accumulator (TMEM lanes 0..127, N columns) is read with tcgen05.ld, one
// row per thread. Every mbarrier wait is bounded; on expiry the CTA records
// an error, waits (bounded) for its last commit, frees its tensor memory and
// skips the epilogue.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include <type_traits>
#include "wait_clock.cuh"

namespace rtm {
namespace tc {

constexpr int kRows = 128;     // M tile
constexpr int kBK = 32;        // K slab per stage
constexpr int kStages = 3;
constexpr int kABytes = kRows * kBK * 2;  // 8 KB
constexpr int kBBytes = 32 * kBK * 2;     // room for N <= 32
constexpr int kStageBytes = kABytes + kBBytes;
constexpr int kTmemCols = 32;
constexpr long long kWaitLimit = 1LL << 24;  // mbarrier polls before giving up
constexpr int kErrTimeout = 5;                // == RTM_ERR_TIMEOUT

// optional per-op extra shared memory (filled once per CTA by Op::load_extra
// and handed to Op::epilogue_x)
template <class Op, class = void>
struct extra_smem {
    static constexpr int value = 0;
};
template <class Op>
struct extra_smem<Op, std::void_t<decltype(Op::kExtraSmem)>> {
    static constexpr int value = Op::kExtraSmem;
};


// byte offset of element (r, k) in a K-major no-swizzle slab (K width 32)
__device__ __forceinline__ uint32_t kmajor_off(int r, int k) {
    return (uint32_t)((r >> 3) * 512 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// store 8 consecutive k values (k % 8 == 0) of row r
__device__ __forceinline__ void st_vec8(uint8_t* slab, int r, int k, uint4 v) {
    *reinterpret_cast<uint4*>(slab + kmajor_off(r, k)) = v;
}
__device__ __forceinline__ void st_one(uint8_t* slab, int r, int k, __nv_bfloat16 v) {
    *reinterpret_cast<__nv_bfloat16*>(slab + kmajor_off(r, k)) = v;
}

__device__ __forceinline__ uint32_t pack2(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);  // .x = a (low half), .y = b
    return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ uint4 pack8(const float* f) {
    return make_uint4(pack2(f[0], f[1]), pack2(f[2], f[3]), pack2(f[4], f[5]), pack2(f[6], f[7]));
}

// shared-memory matrix descriptor (tcgen05): start >> 4 in bits 0-13, leading
// byte offset >> 4 in 16-29, stride byte offset >> 4 in 32-45, the fixed
// version value 1 at bit 46, base offset 0, no swizzle (bits 61-63 = 0)
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor, kind::f16: f32 accumulator (bits 4-5 = 1), bf16 A
// and B (bits 7-9 and 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at
// bit 24
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// bounded wait for the completion of the phase with the given parity
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    const unsigned long long t0 = wait_now();
    for (long long i = 0; i < kWaitLimit; i++) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (wait_expired(i, t0)) break;
    }
    return false;
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// executed by one full warp
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

// 16 consecutive 32-bit columns of this warp's 32 lanes, one lane per thread;
// the wait is in the same statement as the load, so no read of the
// registers can be scheduled before the data is in them
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* out) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) out[i] = __uint_as_float(r[i]);
}

// 16-byte asynchronous global -> shared copy; zero-fills when !valid (the
// source is not read then, but must still be a mapped address)
__device__ __forceinline__ void cp_async16(uint8_t* slab, int r, int k, const void* src, bool valid) {
    const uint32_t dst = smem_u32(slab + kmajor_off(r, k));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                 "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Op interface:
//   using Args;                      kernel arguments
//   static constexpr int N;          16 or 32 output columns
//   static __device__ void tile(const Args&, int& m0, int& c0, int& c1);
//   static __device__ void load(const Args&, int m0, int chunk, uint8_t* sA, uint8_t* sB, int tid);
//   static __device__ void epilogue(const Args&, int m0, int row, const float* acc);
template <class Op>
__global__ void __launch_bounds__(128) k_tc_gemm(const __grid_constant__ typename Op::Args args,
                                                 int* status) {
    constexpr int N = Op::N;
    static_assert(N == 16 || N == 32, "N must be 16 or 32");
    __shared__ __align__(1024) uint8_t smem[kStages][kStageBytes];
    __shared__ __align__(8) uint64_t bars[kStages];
    __shared__ uint32_t tmem_slot;

    const int tid = threadIdx.x, warp = tid >> 5;
    int m0, c0, c1;
    Op::tile(args, m0, c0, c1);
    const int nch = c1 - c0;

    if (tid == 0) {
        for (int s = 0; s < kStages; s++) mbar_init(&bars[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(&tmem_slot, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    constexpr uint32_t idesc = idesc_bf16(kRows, N);

    bool ok = true;
    int issued = 0;
    for (int i = 0; i < nch && ok; i++) {
        const int st = i % kStages;
        if (i >= kStages) ok = mbar_wait(&bars[st], (uint32_t)((i / kStages - 1) & 1));
        // every thread agrees on ok before touching the stage again
        ok = __syncthreads_and(ok);
        if (!ok) break;
        Op::load(args, m0, c0 + i, smem[st], smem[st] + kABytes, tid);
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(smem[st]);
            const uint32_t b0 = a0 + kABytes;
#pragma unroll
            for (int s = 0; s < kBK / 16; s++) {
                mma_bf16(tmem, sdesc(a0 + 256 * s, 128, 512), sdesc(b0 + 256 * s, 128, 512),
                         idesc, (i > 0 || s > 0) ? 1u : 0u);
            }
            mma_commit(&bars[st]);
        }
        issued = i + 1;
    }
    if (issued > 0) {
        const int last = issued - 1;
        const bool done = mbar_wait(&bars[last % kStages], (uint32_t)((last / kStages) & 1));
        ok = ok && done;
    }
    ok = __syncthreads_and(ok);
    tc_fence_after();

    float acc[N];
    if (ok && nch > 0) {
        const uint32_t t = tmem + ((uint32_t)(warp * 32) << 16);
        tmem_ld16(t, acc);
        if constexpr (N == 32) tmem_ld16(t + 16, acc + 16);
    } else {
#pragma unroll
        for (int n = 0; n < N; n++) acc[n] = 0.0f;
    }
    if (ok) Op::epilogue(args, m0, tid, acc);
    else if (tid == 0 && status) atomicCAS(status, 0, kErrTimeout);

    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

}  // namespace tc
}  // namespace rtm

namespace rtm {
namespace tc {

// The same engine with a deeper, asynchronous operand pipeline for ops whose
// A slabs are plain 16-byte gathers: Op::load_async issues cp.async copies
// for A (and stores B synchronously); kAsyncStages slabs are in flight while
// the tensor core works on the oldest. The stage of slab j is refilled only
// after the MMAs of slab j - kAsyncStages have completed (their commit
// mbarrier); every wait is bounded as in k_tc_gemm.
constexpr int kAsyncStages = 4;

template <class Op>
__global__ void __launch_bounds__(128) k_tc_gemm_async(const __grid_constant__ typename Op::Args args,
                                                       int* status) {
    constexpr int N = Op::N;
    constexpr int S = kAsyncStages;
    static_assert(N == 16 || N == 32, "N must be 16 or 32");
    constexpr int L = S - 2;  // slabs loaded ahead; a stage is refilled two MMAs after its use
    __shared__ __align__(1024) uint8_t smem[S][kStageBytes];
    __shared__ __align__(16) uint8_t extra[extra_smem<Op>::value > 0 ? extra_smem<Op>::value : 16];
    __shared__ __align__(8) uint64_t bars[S];
    __shared__ uint32_t tmem_slot;

    const int tid = threadIdx.x, warp = tid >> 5;
    int m0, c0, c1;
    Op::tile(args, m0, c0, c1);
    const int nch = c1 - c0;

    if (tid == 0) {
        for (int s = 0; s < S; s++) mbar_init(&bars[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(&tmem_slot, kTmemCols);
    if constexpr (extra_smem<Op>::value > 0) Op::load_extra(args, extra, tid);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    constexpr uint32_t idesc = idesc_bf16(kRows, N);

    for (int c = 0; c < L; c++) {
        if (c < nch) Op::load_async(args, m0, c0 + c, smem[c], smem[c] + kABytes, tid);
        cp_async_commit();
    }
    bool ok = true;
    int issued = 0;
    for (int i = 0; i < nch && ok; i++) {
        const int j = i + L;
        if (j < nch) {
            // slab j reuses the stage of slab j - S = i - 2, whose MMAs were
            // issued two iterations ago
            if (j >= S) ok = mbar_wait(&bars[(j - S) % S], (uint32_t)(((j - S) / S) & 1));
            ok = __syncthreads_and(ok);
            if (!ok) break;
            Op::load_async(args, m0, c0 + j, smem[j % S], smem[j % S] + kABytes, tid);
        }
        cp_async_commit();
        cp_async_wait<L>();
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const int st = i % S;
            const uint32_t a0 = smem_u32(smem[st]);
            const uint32_t b0 = a0 + kABytes;
#pragma unroll
            for (int s = 0; s < kBK / 16; s++) {
                mma_bf16(tmem, sdesc(a0 + 256 * s, 128, 512), sdesc(b0 + 256 * s, 128, 512),
                         idesc, (i > 0 || s > 0) ? 1u : 0u);
            }
            mma_commit(&bars[st]);
        }
        issued = i + 1;
    }
    cp_async_wait<0>();
    if (issued > 0) {
        const int last = issued - 1;
        const bool done = mbar_wait(&bars[last % S], (uint32_t)((last / S) & 1));
        ok = ok && done;
    }
    ok = __syncthreads_and(ok);
    tc_fence_after();

    float acc[N];
    if (ok && nch > 0) {
        const uint32_t t = tmem + ((uint32_t)(warp * 32) << 16);
        tmem_ld16(t, acc);
        if constexpr (N == 32) tmem_ld16(t + 16, acc + 16);
    } else {
#pragma unroll
        for (int n = 0; n < N; n++) acc[n] = 0.0f;
    }
    if (ok) {
        if constexpr (extra_smem<Op>::value > 0) Op::epilogue_x(args, m0, tid, acc, extra);
        else Op::epilogue(args, m0, tid, acc);
    } else if (tid == 0 && status) {
        atomicCAS(status, 0, kErrTimeout);
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

}  // namespace tc
}  // namespace rtm
