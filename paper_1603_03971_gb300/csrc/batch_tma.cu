// Batched multi-shot RTM with TMA plane loads: the persistent work-queue
// schedule of batch.cu (phase steps of every shot in a wave, per-shot step
// counters, bounded waits) around the plane march of the TMA stencil.
//
// A work item is one tile (TX columns x 16 or 8 rows x a z slab) of one shot
// at one phase step. The block's thread 0 copies each plane with the 3D-in-4D bulk
// tensor copy: the centre plane of u^n with its r-wide halo into a ring of
// P + 1 slots, and, into a second ring, the tile of u^{n-1}, c, the queue head
// (u^n at z + r, no halo) and, on imaging steps, the snapshot and image tiles.
// Each shot's padded fields (c, both field pairs, all checkpoints) sit one
// stride apart in the workspace, and so do its slabs (snapshots, image), so
// three tensor maps per shot (halo tile, plain tile, slab tile) address them
// all through the fourth coordinate. Fields written by other blocks in the
// previous phase step are published by their device-scope fence and counter
// increment; the reading thread acquires the counter and then fences the
// generic proxy against the asynchronous one before its copies read them.
//
// The ring slots and mbarrier phases run on across items: every copy an item
// issues is waited for within the item, so the next item reuses the slots in
// order. Every wait is bounded and shares the abort flag of the launch.

#include <cuda.h>
#include <string.h>

#include "batch_internal.h"
#include "packed_f32x2.cuh"
#include "tma_encode.h"
#include "wait_clock.cuh"

namespace rtm {

namespace {

constexpr long long kPlaneWaitLimit = 1LL << 26;

// tile: 16 threads along x (V points each) by BYT rows (16: 256 threads,
// three blocks per SM; 8: 128 threads, five blocks per SM at radius 4 and
// four at radius 8, where the 8-row tiles keep 4-point vectors)
template <int R, int BYT = 16>
struct BT {
    static constexpr int V = (R == 8 && BYT == 16) ? 2 : 4;  // x points per thread
    static constexpr int BX = 16, BY = BYT;
    static constexpr int TX = V * BX, TY = BY;
    static constexpr int SW = TX + 2 * R, SH = TY + 2 * R;
    static constexpr int HX = R / V;
    static constexpr int P = R == 8 ? 2 : 1;  // planes in flight (three blocks fit per SM)
    static constexpr int NS = P + 1;
    static constexpr int UPLANE = SH * SW, APLANE = TY * TX;
    static constexpr int NAH = 5;  // u^{n-1}, c, queue head, snapshot, image
    static constexpr int SMEM = (NS * UPLANE + NS * NAH * APLANE) * 4;
    static constexpr int G = R == 8 ? (V == 2 ? 4 : 2) : 1;  // queue moves once per G planes
    static constexpr int MINB = BY == 16 ? 3 : (R == 8 ? 4 : 5);
    static_assert(R % 4 == 0 && R % V == 0 && (BY == 16 || BY == 8), "tile");
    static_assert(MINB * (SMEM + 1024 + 1024) <= 228 * 1024, "rings do not fit the resident blocks");
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
__device__ __forceinline__ Vec<V> vld_cg(const float* p) {  // global, coherent at L2
    Vec<V> r;
    if constexpr (V == 4) {
        const float4 t = __ldcg(reinterpret_cast<const float4*>(p));
        r.v[0] = t.x, r.v[1] = t.y, r.v[2] = t.z, r.v[3] = t.w;
    } else {
        const float2 t = __ldcg(reinterpret_cast<const float2*>(p));
        r.v[0] = t.x, r.v[1] = t.y;
    }
    return r;
}
// global store, streaming (evict first): every field a step writes is read
// again only in a later step, after the rest of the wave has gone through L2
template <int V>
__device__ __forceinline__ void vst(float* p, const Vec<V>& a) {
    if constexpr (V == 4)
        __stcs(reinterpret_cast<float4*>(p), make_float4(a.v[0], a.v[1], a.v[2], a.v[3]));
    else
        __stcs(reinterpret_cast<float2*>(p), make_float2(a.v[0], a.v[1]));
}

__device__ __forceinline__ uint32_t s_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
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
// bounded wait; false if it ran out (then the launch's abort flag is raised)
// or if another block already aborted
__device__ __forceinline__ bool bar_wait(uint64_t* b, uint32_t parity, BatchCtrl* ctrl) {
    const uint32_t a = s_u32(b);
    if (bar_poll(a, parity)) return true;  // the common case: the plane is in
    const unsigned long long t0 = wait_now();
    for (long long i = 0; i < kPlaneWaitLimit; i++) {
        if (bar_poll(a, parity)) return true;
        if ((i & 1023) == 1023 && *reinterpret_cast<volatile int*>(&ctrl->abort)) return false;
        if (wait_expired(i, t0)) break;
    }
    atomicExch(&ctrl->abort, 1);
    atomicCAS(&ctrl->status, 0, 5);  // RTM_ERR_TIMEOUT
    return false;
}
// bounded wait that ignores the abort flag: lets the copies already in
// flight land before an aborting block leaves
__device__ __forceinline__ void bar_drain(uint64_t* b, uint32_t parity) {
    const uint32_t a = s_u32(b);
    const unsigned long long t0 = wait_now();
    for (long long i = 0; i < kPlaneWaitLimit; i++)
        if (bar_poll(a, parity) || wait_expired(i, t0)) return;
}
__device__ __forceinline__ void bar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_u32(b)) : "memory");
}
__device__ __forceinline__ void tma4(float* dst, const CUtensorMap* map, int x, int y, int z,
                                     int f, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(s_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(f), "r"(s_u32(bar))
        : "memory");
}

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// bounded wait for *counter >= target; false if it ran out or another block aborted
__device__ bool wait_counter(BatchCtrl* ctrl, const unsigned int* counter, unsigned int target,
                             long long timeout_cycles, int* status) {
    const long long t0 = clock64();
    while (ld_acquire(counter) < target) {
        if (*reinterpret_cast<volatile int*>(&ctrl->abort)) return false;
        if (clock64() - t0 > timeout_cycles) {
            atomicExch(&ctrl->abort, 1);
            atomicCAS(&ctrl->status, 0, 5);  // RTM_ERR_TIMEOUT
            if (status) atomicCAS(status, 0, 5);
            return false;
        }
        __nanosleep(64);
    }
    return true;
}

// ring position shared by the block: slot and mbarrier phase of the next
// plane to wait for (every thread) and slot of the next plane to copy
// (thread 0)
struct RingPos {
    int slot, phase, issue;
};

// field indices in a shot's field stack
constexpr int F_C = 0, F_F0 = 1, F_F1 = 2, F_M0 = 3, F_M1 = 4, F_CK = 5;

template <int R, int BY>
__device__ bool item_tma(const BatchTmaArgs& T, const BatchShot& S, const BatchPhase ph, int tile,
                         int s, float* uring, float* aring, uint64_t* ubar, uint64_t* abar,
                         RingPos& rp) {
    using B = BT<R, BY>;
    constexpr int V = B::V;
    using VT = Vec<V>;
    const BatchArgs& A = T.a;
    const CUtensorMap* mU = &T.maps[s][0];
    const CUtensorMap* mP = &T.maps[s][1];
    const CUtensorMap* mS = &T.maps[s][2];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * B::BX + tx;
    const int bx = tile % S.tiles_x;
    const int by = (tile / S.tiles_x) % S.tiles_y;
    const int bz = tile / (S.tiles_x * S.tiles_y);
    const int x0 = bx * B::TX, y0 = by * B::TY;
    const int x = x0 + V * tx, y = y0 + ty;
    const int zb = bz * A.zchunk;
    const int ze = min(S.NZ, zb + A.zchunk);
    const bool own = x < S.NX && y < S.NY;
    const size_t plane = (size_t)S.NX * S.NY;
    const size_t col = (size_t)y * S.NX + x;

    // buffers of this phase step (pointers for the stores, stack indices for the copies)
    int icur, iprev;
    bool zero_in = false;
    float* ck_a = nullptr;  // forward: checkpoint destinations
    float* ck_b = nullptr;
    float* snap_w = nullptr;  // recompute: snapshot to write
    int snap_r = -1;          // backward: slab of the snapshot to image with
    if (ph.kind == PH_FWD) {
        const int n = ph.step;
        icur = (n & 1) ? F_F0 : F_F1;
        iprev = (n & 1) ? F_F1 : F_F0;
        zero_in = (n == 0);
        if ((n + 1) % A.ckpt_every == 0 && n + 1 < A.nt) {
            const size_t j = (size_t)((n + 1) / A.ckpt_every);
            ck_a = S.ckpt + ((j - 1) * 2 + 0) * S.fstride;
            ck_b = S.ckpt + ((j - 1) * 2 + 1) * S.fstride;
        }
    } else if (ph.kind == PH_REC) {
        int ia, ib;
        if (ph.seg == 0) {
            ia = F_F0;
            ib = F_F1;
            zero_in = (ph.local == 0);
        } else {
            ia = F_CK + (ph.seg - 1) * 2;
            ib = ia + 1;
        }
        icur = (ph.local & 1) ? ia : ib;
        iprev = (ph.local & 1) ? ib : ia;
        if ((ph.step + 1) % A.image_every == 0) snap_w = S.snap + (size_t)ph.local * S.sstride;
    } else {
        const int bi = A.nt - ph.step;  // 0 for m = nt
        icur = (bi & 1) ? F_M0 : F_M1;
        iprev = (bi & 1) ? F_M1 : F_M0;
        zero_in = (ph.step == A.nt);
        if (ph.step % A.image_every == 0) snap_r = ph.local;
    }
    const float* cur = S.c + (size_t)icur * S.fstride;
    float* prev = const_cast<float*>(S.c) + (size_t)iprev * S.fstride;
    // zero inputs: the first step of a recursion reads nothing and clears the
    // buffer that holds the step before it
    float* clear = zero_in ? const_cast<float*>(cur) : nullptr;
    const bool rd = own && !zero_in;
    const int img_slab = A.ckpt_every;

    const bool xm = (x + V - 1 >= S.nb) && (x < S.nb + S.nx);
    const bool ym = (y >= S.nb) && (y < S.nb + S.ny);
    const size_t slab_col = (size_t)(y - S.nb) * S.NX + x;
    const size_t slab_plane = (size_t)S.ny * S.NX;

    // copies of plane p: centre plane of u^n with halo; the tiles of u^{n-1},
    // c and the queue head (u^n at p + r); the snapshot and image tiles
    const uint32_t abytes =
        (uint32_t)((zero_in ? 1 : 3) + (snap_r >= 0 ? 2 : 0)) * B::APLANE * 4;
    int nissued = 0;  // planes of this item copied (thread 0)
    auto issue = [&](int p) {
        const int sl = rp.issue;
        float* abase = aring + sl * B::NAH * B::APLANE;
        if (!zero_in) {
            bar_expect(&ubar[sl], B::UPLANE * 4);
            tma4(uring + sl * B::UPLANE, mU, x0 - R, y0 - R, p, icur, &ubar[sl]);
        } else {
            bar_arrive(&ubar[sl]);  // no halo plane: complete the phase, keep the rings in step
        }
        bar_expect(&abar[sl], abytes);
        tma4(abase + B::APLANE, mP, x0, y0, p, F_C, &abar[sl]);
        if (!zero_in) {
            tma4(abase, mP, x0, y0, p, iprev, &abar[sl]);
            tma4(abase + 2 * B::APLANE, mP, x0, y0, p + R, icur, &abar[sl]);
        }
        if (snap_r >= 0) {
            tma4(abase + 3 * B::APLANE, mS, x0, y0 - S.nb, p - S.nb, snap_r, &abar[sl]);
            tma4(abase + 4 * B::APLANE, mS, x0, y0 - S.nb, p - S.nb, img_slab, &abar[sl]);
        }
        rp.issue = sl + 1 == B::NS ? 0 : sl + 1;
        nissued++;
    };
    const int slot0 = rp.slot, phase0 = rp.phase;
    if (tid == 0) {
        // the previous phase step's fields were written through the generic
        // proxy (acquired with the counter); order them before the copies
        asm volatile("fence.proxy.async.global;" ::: "memory");
        for (int p = zb; p < zb + B::P && p < ze; p++) issue(p);
    }

    Vec<V> gxy = vzero<V>();
    if (own) {
        const float gyv = S.gy[y];
#pragma unroll
        for (int i = 0; i < V; i++) gxy.v[i] = S.gx[x + i] * gyv;
    }
    // queue: plane z0 + t of a group reads entries t .. t + 2r (head 2r + t)
    constexpr int G = B::G;
    VT q[2 * R + G];
#pragma unroll
    for (int i = 0; i < 2 * R; i++) {
        const int zz = zb - R + i;
        q[i] = (rd && zz >= 0 && zz < S.NZ) ? vld_cg<V>(cur + (size_t)zz * plane + col)
                                            : vzero<V>();
    }
#pragma unroll
    for (int i = 2 * R; i < 2 * R + G; i++) q[i] = vzero<V>();

    const bool do_src = ph.kind != PH_BWD;
    const float w = do_src ? A.wavelet[ph.step] : 0.f;
    const int own_off = (R + ty) * B::SW + R + V * tx;
    const int aux_off = ty * B::TX + V * tx;
    bool ok = true;  // the same in every thread (block-wide vote each plane)
    int nwaited = 0;

    for (int z0 = zb; z0 < ze && ok; z0 += G) {
#pragma unroll
        for (int t = 0; t < G; t++) {
            const int z = z0 + t;
            if (z >= ze || !ok) break;  // the same for every thread of the block
            const int sl = rp.slot;
            bool got = bar_wait(&ubar[sl], (uint32_t)rp.phase, A.ctrl);
            got = bar_wait(&abar[sl], (uint32_t)rp.phase, A.ctrl) && got;
            // block-wide vote; also every thread is past plane z - 1, whose
            // slots plane z + P reuses
            ok = __syncthreads_and(got) != 0;
            if (!ok) break;
            nwaited++;
            if (tid == 0 && z + B::P < ze) issue(z + B::P);
            const float* Sm = uring + sl * B::UPLANE;
            const float* aux = aring + sl * B::NAH * B::APLANE;
            q[2 * R + t] = zero_in ? vzero<V>() : vlds<V>(aux + 2 * B::APLANE + aux_off);

            if (own) {
                VT lap = vzero<V>();
                if (!zero_in) {
                    float v[V + 2 * R];
#pragma unroll
                    for (int h = 0; h < B::HX; h++) {
                        const VT l = vlds<V>(Sm + (R + ty) * B::SW + V * tx + V * h);
                        const VT r = vlds<V>(Sm + (R + ty) * B::SW + R + V * tx + V + V * h);
#pragma unroll
                        for (int i = 0; i < V; i++) {
                            v[V * h + i] = l.v[i];
                            v[R + V + V * h + i] = r.v[i];
                        }
                    }
#pragma unroll
                    for (int i = 0; i < V; i++) v[R + i] = q[R + t].v[i];
                    // the Laplacian on packed point pairs (f32x2); radius 8
                    // sums even and odd offsets in two chains, then adds
                    namespace P2 = f32x2;
                    uint64_t L2[V / 2], L2o[V / 2];
                    const uint64_t a0 = P2::pack(A.a[0], A.a[0]);
#pragma unroll
                    for (int j = 0; j < V / 2; j++) {
                        L2[j] = P2::mul(a0, P2::pack(q[R + t].v[2 * j], q[R + t].v[2 * j + 1]));
                        L2o[j] = 0;  // two +0.0f
                    }
#pragma unroll
                    for (int k = 1; k <= R; k++) {
                        const VT ym_ = vlds<V>(Sm + (R + ty - k) * B::SW + R + V * tx);
                        const VT yp_ = vlds<V>(Sm + (R + ty + k) * B::SW + R + V * tx);
                        const uint64_t ak = P2::pack(A.a[k], A.a[k]);
#pragma unroll
                        for (int j = 0; j < V / 2; j++) {
                            const int i = 2 * j;
                            const uint64_t px = P2::add(P2::pack(v[R + i - k], v[R + i + 1 - k]),
                                                        P2::pack(v[R + i + k], v[R + i + 1 + k]));
                            const uint64_t py = P2::add(P2::pack(ym_.v[i], ym_.v[i + 1]),
                                                        P2::pack(yp_.v[i], yp_.v[i + 1]));
                            const uint64_t pz =
                                P2::add(P2::pack(q[R + t - k].v[i], q[R + t - k].v[i + 1]),
                                        P2::pack(q[R + t + k].v[i], q[R + t + k].v[i + 1]));
                            if (R == 8 && (k & 1))
                                L2o[j] = P2::fma(ak, P2::add(P2::add(px, py), pz), L2o[j]);
                            else
                                L2[j] = P2::fma(ak, P2::add(P2::add(px, py), pz), L2[j]);
                        }
                    }
#pragma unroll
                    for (int j = 0; j < V / 2; j++) {
                        if (R == 8)
                            P2::unpack(P2::add(L2[j], L2o[j]), lap.v[2 * j], lap.v[2 * j + 1]);
                        else
                            P2::unpack(L2[j], lap.v[2 * j], lap.v[2 * j + 1]);
                    }
                }
                const VT up = zero_in ? vzero<V>() : vlds<V>(aux + aux_off);
                const VT cc = vlds<V>(aux + B::APLANE + aux_off);
                const VT& qc = q[R + t];
                const float gzv = S.gz[z];
                VT out;
#pragma unroll
                for (int i = 0; i < V; i++) {
                    const float g = gxy.v[i] * gzv;
                    out.v[i] = g * fmaf(cc.v[i], lap.v[i], 2.0f * qc.v[i]) - (g * g) * up.v[i];
                }
                // source injection: u^{n+1}[s] += c_s w^n / dx^3
                if (do_src && z == S.src_z && y == S.src_y && S.src_x >= x && S.src_x < x + V)
                    out.v[S.src_x - x] += cc.v[S.src_x - x] * w * A.inv_dx3;
                const bool rplane = (z == S.rec_z) && ym;
                if (ph.kind == PH_BWD && rplane) {
                    // adjoint injection: mu^m[rec] += c g r^{m-1} / dx^3
                    const float* row =
                        S.dobs + ((size_t)(ph.step - 1) * S.ny + (y - S.nb)) * S.nx;
#pragma unroll
                    for (int i = 0; i < V; i++) {
                        const int xi = x + i - S.nb;
                        if (xi >= 0 && xi < S.nx)
                            out.v[i] += cc.v[i] * (gxy.v[i] * gzv) * row[xi] * A.inv_dx3;
                    }
                }
                const size_t o = (size_t)z * plane + col;
                vst<V>(prev + o, out);
                if (clear) vst<V>(clear + o, vzero<V>());
                if (ck_a) {
                    vst<V>(ck_a + o, qc);
                    vst<V>(ck_b + o, out);
                }
                const bool inm = xm && ym && z >= S.nb && z < S.nb + S.nz;
                if (inm) {
                    const size_t so = (size_t)(z - S.nb) * slab_plane + slab_col;
                    if (snap_w) vst<V>(snap_w + so, out);
                    if (snap_r >= 0) {
                        const VT sv = vlds<V>(aux + 3 * B::APLANE + aux_off);
                        VT iv = vlds<V>(aux + 4 * B::APLANE + aux_off);
#pragma unroll
                        for (int i = 0; i < V; i++) iv.v[i] = fmaf(sv.v[i], out.v[i], iv.v[i]);
                        vst<V>(S.img + so, iv);
                    }
                }
                if (ph.kind == PH_FWD && rplane && S.data) {
                    float* row = S.data + ((size_t)ph.step * S.ny + (y - S.nb)) * S.nx;
#pragma unroll
                    for (int i = 0; i < V; i++) {
                        const int xi = x + i - S.nb;
                        if (xi >= 0 && xi < S.nx) row[xi] = out.v[i];
                    }
                }
            }
            if (++rp.slot == B::NS) rp.slot = 0, rp.phase ^= 1;
        }
#pragma unroll
        for (int i = 0; i < 2 * R; i++) q[i] = q[i + G];
    }
    if (!ok && tid == 0) {
        // copies still in flight must land before the block leaves
        for (int j = nwaited; j < nissued; j++) {
            const int k = slot0 + j;
            const int sl = k % B::NS;
            const uint32_t ph = (uint32_t)(phase0 ^ ((k / B::NS) & 1));
            bar_drain(&ubar[sl], ph);
            bar_drain(&abar[sl], ph);
        }
    }
    return ok;
}

template <int R, int BY>
__global__ void __launch_bounds__(16 * BY, BT<R, BY>::MINB)
    k_batch_tma(const __grid_constant__ BatchTmaArgs T) {
    using B = BT<R, BY>;
    extern __shared__ __align__(128) float dsm[];
    float* uring = dsm;
    float* aring = dsm + B::NS * B::UPLANE;
    __shared__ __align__(8) uint64_t ubar[B::NS];
    __shared__ __align__(8) uint64_t abar[B::NS];
    __shared__ long long s_item;
    __shared__ int s_go, s_shot_i;
    // the item's shot, copied once per item: its fields are read again in
    // every plane, and shared-memory reads of them are cheaper than global
    // ones that each store of the plane before may have overwritten
    __shared__ BatchShot s_shot;
    const BatchArgs& A = T.a;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    if (tid == 0) {
        for (int i = 0; i < B::NS; i++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_u32(&ubar[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_u32(&abar[i])));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    RingPos rp{0, 0, 0};
    const long long total = A.items_per_phase * (long long)A.nphases;
    for (;;) {
        if (tid == 0) s_item = (long long)atomicAdd(&A.ctrl->next, 1ull);
        __syncthreads();
        const long long item = s_item;
        if (item >= total) break;
        const int t = (int)(item / A.items_per_phase);
        const long long r = item % A.items_per_phase;
        if (tid == 0) {
            int s = 0;
            while (s + 1 < A.nshots && A.shots[s + 1].item_base <= r) s++;
            s_shot = A.shots[s];
            s_shot_i = s;
            const int tile = (int)(r - A.shots[s].item_base);
            unsigned int target = (unsigned int)t * (unsigned int)A.shots[s].ntiles;
            if (s == A.poison_shot && t == 0 && tile == 0) target = 0xFFFFFFFFu;  // failure test
            s_go = wait_counter(A.ctrl, &A.ctrl->done[s], target, A.timeout_cycles, A.status) ? 1
                                                                                         : 0;
        }
        __syncthreads();
        if (!s_go) break;
        const int s = s_shot_i;
        const BatchShot& S = s_shot;
        const int tile = (int)(r - S.item_base);
        const bool ok = item_tma<R, BY>(T, S, A.phases[t], tile, s, uring, aring, ubar, abar, rp);
        __threadfence();
        __syncthreads();
        if (!ok) {
            if (tid == 0 && A.status) atomicCAS(A.status, 0, 5);
            break;
        }
        if (tid == 0) atomicAdd(&A.ctrl->done[s], 1u);
    }
}

}  // namespace

// dispatch on (radius, tile rows)
template <class F>
cudaError_t with_tile(int radius, int tile_rows, F&& f) {
    if (radius == 4 && tile_rows == 16) return f(BT<4, 16>(), k_batch_tma<4, 16>);
    if (radius == 4 && tile_rows == 8) return f(BT<4, 8>(), k_batch_tma<4, 8>);
    if (radius == 8 && tile_rows == 16) return f(BT<8, 16>(), k_batch_tma<8, 16>);
    if (radius == 8 && tile_rows == 8) return f(BT<8, 8>(), k_batch_tma<8, 8>);
    return cudaErrorInvalidValue;
}

int batch_tma_tile_x(int radius, int tile_rows) {
    int tx = 0;
    with_tile(radius, tile_rows, [&](auto b, auto) {
        tx = decltype(b)::TX;
        return cudaSuccess;
    });
    return tx;
}

int batch_tma_blocks_per_sm(int radius, int tile_rows) {
    int n = 0;
    const cudaError_t e = with_tile(radius, tile_rows, [&](auto b, auto kernel) {
        using B = decltype(b);
        cudaError_t r = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             B::SMEM);
        if (r != cudaSuccess) return r;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, 16 * B::BY, B::SMEM);
    });
    return e == cudaSuccess ? n : 0;
}

// the three tensor maps of one shot: halo tile and plain tile over its field
// stack, plain tile over its slab stack
cudaError_t batch_tma_maps(int radius, int tile_rows, const BatchShot& b, int nfields,
                           int nslabs, CUtensorMap* maps) {
    EncodeTiledFn f = tma_encoder();
    if (!f) return cudaErrorNotSupported;
    const int TX = batch_tma_tile_x(radius, tile_rows);
    const int TY = tile_rows;
    if (TX == 0) return cudaErrorInvalidValue;
    const cuuint64_t fd[4] = {(cuuint64_t)b.NX, (cuuint64_t)b.NY, (cuuint64_t)b.NZ,
                              (cuuint64_t)nfields};
    const cuuint64_t fs[3] = {(cuuint64_t)b.NX * 4, (cuuint64_t)b.NX * b.NY * 4,
                              (cuuint64_t)b.fstride * 4};
    const cuuint64_t sd[4] = {(cuuint64_t)b.NX, (cuuint64_t)b.ny, (cuuint64_t)b.nz,
                              (cuuint64_t)nslabs};
    const cuuint64_t ss[3] = {(cuuint64_t)b.NX * 4, (cuuint64_t)b.NX * b.ny * 4,
                              (cuuint64_t)b.sstride * 4};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const cuuint32_t boxU[4] = {(cuuint32_t)(TX + 2 * radius), (cuuint32_t)(TY + 2 * radius), 1, 1};
    const cuuint32_t boxP[4] = {(cuuint32_t)TX, (cuuint32_t)TY, 1, 1};
    if (f(&maps[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(b.c), fd, fs, boxU,
          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    if (f(&maps[1], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(b.c), fd, fs, boxP,
          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    if (f(&maps[2], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, b.snap, sd, ss, boxP, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    return cudaSuccess;
}

cudaError_t launch_batch_tma(int radius, int tile_rows, const BatchTmaArgs& a, int grid,
                             cudaStream_t s) {
    return with_tile(radius, tile_rows, [&](auto b, auto kernel) {
        using B = decltype(b);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(16, B::BY);
        cfg.dynamicSmemBytes = B::SMEM;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, kernel, a);
    });
}

}  // namespace rtm
