// Batched multi-shot RTM in one persistent, cooperative launch.
//
// Every shot of a wave runs the same schedule of 3 nt phase steps on its own
// padded aperture grid: nt forward steps (fused source injection, receiver
// gather, checkpoint writes), then for each checkpoint segment, last first,
// its recompute steps (in place in the checkpoint slot, fused snapshot
// writes) and its backward steps (fused adjoint injection at the receiver
// plane and zero-lag imaging). A work item is one tile (64 x 16 columns x a
// z slab) of one shot at one phase step; items are ordered by (phase step,
// shot, tile) and handed out by an atomic queue head, so blocks that finish
// early take the next item of any shot (the GPU form of the dynamic tile
// schedule of the paper, Sec. III). Before an item starts, the block waits
// until all tiles of the same shot's previous phase step are done (a
// per-shot counter; bounded wait with a shared abort flag). Items are
// claimed in order and only wait on earlier items of resident blocks, so
// the schedule cannot deadlock.
//
// Fields written and read within the launch are loaded through L2
// (ld.global.cg); each block publishes its stores with a device-scope fence
// before it increments the shot's counter.

#include "batch_internal.h"
#include "packed_f32x2.cuh"
#include "stencil_common.cuh"

namespace rtm {

namespace {

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_volatile_int(const int* p) {
    return *reinterpret_cast<const volatile int*>(p);
}

// bounded wait for *counter >= target; false if it ran out or another block aborted
__device__ bool wait_counter(BatchCtrl* ctrl, const unsigned int* counter, unsigned int target,
                             long long timeout_cycles, int* status) {
    const long long t0 = clock64();
    while (ld_acquire(counter) < target) {
        if (ld_volatile_int(&ctrl->abort)) return false;
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

template <int R>
__device__ void process_item(const BatchArgs& A, const BatchShot& S, const BatchPhase ph,
                             int tile, float (*sm)[Tile<R>::SH][Tile<R>::SW]) {
    using T = Tile<R>;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int bx = tile % S.tiles_x;
    const int by = (tile / S.tiles_x) % S.tiles_y;
    const int bz = tile / (S.tiles_x * S.tiles_y);
    const int x0 = bx * T::TX, y0 = by * T::TY;
    const int x = x0 + 4 * tx, y = y0 + ty;
    const int zb = bz * A.zchunk;
    const int ze = min(S.NZ, zb + A.zchunk);
    const bool xin = x < S.NX, yin = y < S.NY, own = xin && yin;
    const size_t plane = (size_t)S.NX * S.NY;
    const size_t col = (size_t)y * S.NX + x;

    // buffers of this phase step
    const float* cur;
    float* prev;
    bool zero_in = false;
    float* ck_a = nullptr;  // forward: checkpoint destinations
    float* ck_b = nullptr;
    float* snap_w = nullptr;  // recompute: snapshot to write
    const float* snap_r = nullptr;  // backward: snapshot to image with
    if (ph.kind == PH_FWD) {
        const int n = ph.step;
        cur = (n & 1) ? S.f0 : S.f1;
        prev = (n & 1) ? S.f1 : S.f0;
        zero_in = (n == 0);
        if ((n + 1) % A.ckpt_every == 0 && n + 1 < A.nt) {
            const size_t j = (size_t)((n + 1) / A.ckpt_every);
            ck_a = S.ckpt + ((j - 1) * 2 + 0) * S.fstride;
            ck_b = S.ckpt + ((j - 1) * 2 + 1) * S.fstride;
        }
    } else if (ph.kind == PH_REC) {
        float *a, *b;
        if (ph.seg == 0) {
            a = S.f0;
            b = S.f1;
            zero_in = (ph.local == 0);
        } else {
            a = S.ckpt + ((size_t)(ph.seg - 1) * 2 + 0) * S.fstride;
            b = S.ckpt + ((size_t)(ph.seg - 1) * 2 + 1) * S.fstride;
        }
        cur = (ph.local & 1) ? a : b;
        prev = (ph.local & 1) ? b : a;
        if ((ph.step + 1) % A.image_every == 0)
            snap_w = S.snap + (size_t)ph.local * S.sstride;
    } else {
        const int bi = A.nt - ph.step;  // 0 for m = nt
        cur = (bi & 1) ? S.m0 : S.m1;
        prev = (bi & 1) ? S.m1 : S.m0;
        zero_in = (ph.step == A.nt);
        if (ph.step % A.image_every == 0)
            snap_r = S.snap + (size_t)ph.local * S.sstride;
    }
    // zero inputs: the first step of a recursion reads nothing and clears the
    // buffer that holds the step before it
    float* clear = zero_in ? const_cast<float*>(cur) : nullptr;

    const bool hx_left = tx < T::HX;
    const bool hx_right = tx >= T::BX - T::HX;
    const int hx_x = hx_left ? (x0 - R + 4 * tx) : (x0 + T::TX + 4 * (tx - (T::BX - T::HX)));
    const bool hx_ok = !zero_in && (hx_left || hx_right) && yin && hx_x >= 0 && hx_x < S.NX;
    const size_t hx_col = (size_t)y * S.NX + (hx_ok ? hx_x : 0);
    const int hx_sc = hx_left ? 4 * tx : (R + T::TX + 4 * (tx - (T::BX - T::HX)));
    const bool hy_top = ty < R;
    const bool hy_bot = ty >= T::TY - R;
    const int hy_y = hy_top ? (y0 - R + ty) : (y0 + R + ty);
    const bool hy_ok = !zero_in && (hy_top || hy_bot) && xin && hy_y >= 0 && hy_y < S.NY;
    const size_t hy_col = (size_t)(hy_ok ? hy_y : 0) * S.NX + x;
    const int hy_sr = hy_top ? ty : ty + 2 * R;

    const bool xm = (x + 3 >= S.nb) && (x < S.nb + S.nx);
    const bool ym = (y >= S.nb) && (y < S.nb + S.ny);
    const size_t slab_col = (size_t)(y - S.nb) * S.NX + x;
    const size_t slab_plane = (size_t)S.ny * S.NX;
    const bool rd = own && !zero_in;

    F4 gxy = zero4();
    if (own) {
        const float gyv = S.gy[y];
#pragma unroll
        for (int i = 0; i < 4; i++) gxy.v[i] = S.gx[x + i] * gyv;
    }
    // the z loop runs in groups of U planes: step t reads its centre as
    // q[R + t] and prefetches the next head into q[2R + t + 1]; the queue
    // moves by U once per group (2R / U register moves per plane)
    constexpr int U = (R == 8) ? 4 : 1;
    F4 q[2 * R + U + 1];
#pragma unroll
    for (int i = 0; i < 2 * R + 1; i++) {
        const int zz = zb - R + i;
        q[i] = (rd && zz >= 0 && zz < S.NZ) ? ld_l2(cur + (size_t)zz * plane + col) : zero4();
    }
#pragma unroll
    for (int i = 2 * R + 1; i < 2 * R + U + 1; i++) q[i] = zero4();
    F4 hxv = hx_ok ? ld_l2(cur + (size_t)zb * plane + hx_col) : zero4();
    F4 hyv = hy_ok ? ld_l2(cur + (size_t)zb * plane + hy_col) : zero4();
    F4 up = rd ? ld_l2(prev + (size_t)zb * plane + col) : zero4();
    F4 cc = own ? ld_keep(S.c + (size_t)zb * plane + col) : zero4();

    const bool do_src = ph.kind != PH_BWD;
    const float w = do_src ? A.wavelet[ph.step] : 0.f;

    for (int zg = zb; zg < ze; zg += U) {
#pragma unroll
    for (int t = 0; t < U; t++) {
        const int z = zg + t;
        if (z >= ze) break;  // the same for every thread of the block
        float(*Sm)[T::SW] = sm[(z - zb) & 1];
        sts4(&Sm[R + ty][R + 4 * tx], q[R + t]);
        if (hx_left || hx_right) sts4(&Sm[R + ty][hx_sc], hxv);
        if (hy_top || hy_bot) sts4(&Sm[hy_sr][R + 4 * tx], hyv);
        const int zn = z + 1;
        F4 qn = zero4(), hxn = zero4(), hyn = zero4(), upn = zero4(), ccn = zero4();
        if (zn < ze) {
            const int zq = zn + R;
            if (rd && zq < S.NZ) qn = ld_l2(cur + (size_t)zq * plane + col);
            if (hx_ok) hxn = ld_l2(cur + (size_t)zn * plane + hx_col);
            if (hy_ok) hyn = ld_l2(cur + (size_t)zn * plane + hy_col);
            if (rd) upn = ld_l2(prev + (size_t)zn * plane + col);
            if (own) ccn = ld_keep(S.c + (size_t)zn * plane + col);
        }
        __syncthreads();
        if (own) {
            float v[4 + 2 * R];
#pragma unroll
            for (int h = 0; h < T::HX; h++) {
                const F4 l = lds4(&Sm[R + ty][4 * tx + 4 * h]);
                const F4 r = lds4(&Sm[R + ty][R + 4 * tx + 4 + 4 * h]);
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    v[4 * h + i] = l.v[i];
                    v[R + 4 + 4 * h + i] = r.v[i];
                }
            }
#pragma unroll
            for (int i = 0; i < 4; i++) v[R + i] = q[R + t].v[i];
            // the Laplacian on packed point pairs (f32x2), in the scalar
            // form's order of sums
            F4 lap;
            {
                namespace P2 = f32x2;
                uint64_t L2[2];
                const uint64_t a0 = P2::pack(A.a[0], A.a[0]);
#pragma unroll
                for (int j = 0; j < 2; j++)
                    L2[j] = P2::mul(a0, P2::pack(q[R + t].v[2 * j], q[R + t].v[2 * j + 1]));
#pragma unroll
                for (int k = 1; k <= R; k++) {
                    const F4 ym_ = lds4(&Sm[R + ty - k][R + 4 * tx]);
                    const F4 yp_ = lds4(&Sm[R + ty + k][R + 4 * tx]);
                    const uint64_t ak = P2::pack(A.a[k], A.a[k]);
#pragma unroll
                    for (int j = 0; j < 2; j++) {
                        const int i = 2 * j;
                        const uint64_t px = P2::add(P2::pack(v[R + i - k], v[R + i + 1 - k]),
                                                    P2::pack(v[R + i + k], v[R + i + 1 + k]));
                        const uint64_t py = P2::add(P2::pack(ym_.v[i], ym_.v[i + 1]),
                                                    P2::pack(yp_.v[i], yp_.v[i + 1]));
                        const uint64_t pz =
                            P2::add(P2::pack(q[R + t - k].v[i], q[R + t - k].v[i + 1]),
                                    P2::pack(q[R + t + k].v[i], q[R + t + k].v[i + 1]));
                        L2[j] = P2::fma(ak, P2::add(P2::add(px, py), pz), L2[j]);
                    }
                }
#pragma unroll
                for (int j = 0; j < 2; j++) P2::unpack(L2[j], lap.v[2 * j], lap.v[2 * j + 1]);
            }
            const float gzv = S.gz[z];
            F4 out;
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const float g = gxy.v[i] * gzv;
                out.v[i] = g * fmaf(cc.v[i], lap.v[i], 2.0f * q[R + t].v[i]) - (g * g) * up.v[i];
            }
            // source injection: u^{n+1}[s] += c_s w^n / dx^3
            if (do_src && z == S.src_z && y == S.src_y && S.src_x >= x && S.src_x < x + 4)
                out.v[S.src_x - x] += cc.v[S.src_x - x] * w * A.inv_dx3;
            const bool rplane = (z == S.rec_z) && ym;
            if (ph.kind == PH_BWD && rplane) {
                // adjoint injection: mu^m[rec] += c g r^{m-1} / dx^3
                const float* row = S.dobs + ((size_t)(ph.step - 1) * S.ny + (y - S.nb)) * S.nx;
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    const int xi = x + i - S.nb;
                    if (xi >= 0 && xi < S.nx)
                        out.v[i] += cc.v[i] * (gxy.v[i] * gzv) * row[xi] * A.inv_dx3;
                }
            }
            const size_t o = (size_t)z * plane + col;
            st_plain4(prev + o, out);
            if (clear) st_plain4(clear + o, zero4());
            if (ck_a) {
                st_plain4(ck_a + o, q[R + t]);
                st_plain4(ck_b + o, out);
            }
            const bool inm = xm && ym && z >= S.nb && z < S.nb + S.nz;
            if (inm) {
                const size_t so = (size_t)(z - S.nb) * slab_plane + slab_col;
                if (snap_w) st_plain4(snap_w + so, out);
                if (snap_r) {
                    const F4 sv = ld_l2(snap_r + so);
                    F4 iv = ld_l2(S.img + so);
#pragma unroll
                    for (int i = 0; i < 4; i++) iv.v[i] = fmaf(sv.v[i], out.v[i], iv.v[i]);
                    st_plain4(S.img + so, iv);
                }
            }
            if (ph.kind == PH_FWD && rplane && S.data) {
                float* row = S.data + ((size_t)ph.step * S.ny + (y - S.nb)) * S.nx;
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    const int xi = x + i - S.nb;
                    if (xi >= 0 && xi < S.nx) row[xi] = out.v[i];
                }
            }
        }
        q[2 * R + t + 1] = qn;
        hxv = hxn;
        hyv = hyn;
        up = upn;
        cc = ccn;
    }
#pragma unroll
        for (int i = 0; i <= 2 * R; i++) q[i] = q[i + U];
    }
}

template <int R>
__global__ void __launch_bounds__(256, R == 4 ? 2 : 1) k_batch(const __grid_constant__ BatchArgs A) {
    using T = Tile<R>;
    __shared__ __align__(16) float sm[2][T::SH][T::SW];
    __shared__ long long s_item;
    __shared__ int s_go;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const long long total = A.items_per_phase * (long long)A.nphases;
    for (;;) {
        if (tid == 0) s_item = (long long)atomicAdd(&A.ctrl->next, 1ull);
        __syncthreads();
        const long long item = s_item;
        if (item >= total) break;
        const int t = (int)(item / A.items_per_phase);
        const long long r = item % A.items_per_phase;
        int s = 0;
        while (s + 1 < A.nshots && A.shots[s + 1].item_base <= r) s++;
        const BatchShot& S = A.shots[s];
        const int tile = (int)(r - S.item_base);
        if (tid == 0) {
            unsigned int target = (unsigned int)t * (unsigned int)S.ntiles;
            if (s == A.poison_shot && t == 0 && tile == 0) target = 0xFFFFFFFFu;  // failure test
            s_go = wait_counter(A.ctrl, &A.ctrl->done[s], target, A.timeout_cycles, A.status) ? 1
                                                                                         : 0;
        }
        __syncthreads();
        if (!s_go) break;
        process_item<R>(A, S, A.phases[t], tile, sm);
        __threadfence();
        __syncthreads();
        if (tid == 0) atomicAdd(&A.ctrl->done[s], 1u);
    }
}

// c of one shot: its aperture of the full model, edge-padded by nb; and the
// sponge profiles of its padded grid
__global__ void k_batch_prep(BatchShot S, const float* __restrict__ vel, int fnx, int fny, int ox,
                             int oy, int oz, float dt2, float* c, float* gx, float* gy, float* gz) {
    const long long N = (long long)S.NX * S.NY * S.NZ;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % S.NX);
        const int y = (int)((i / S.NX) % S.NY);
        const int z = (int)(i / ((long long)S.NX * S.NY));
        const int mx = min(max(x - S.nb, 0), S.nx - 1) + ox;
        const int my = min(max(y - S.nb, 0), S.ny - 1) + oy;
        const int mz = min(max(z - S.nb, 0), S.nz - 1) + oz;
        const float v = vel[((long long)mz * fny + my) * fnx + mx];
        c[i] = v * v * dt2;
        if (i < S.NX || i < S.NY || i < S.NZ) {
            const int j = (int)i;
            auto prof = [&](int n) {
                const int d = min(j, n - 1 - j);
                if (d >= S.nb) return 1.0f;
                const double a = 0.015 * (double)(S.nb - d);
                return (float)exp(-a * a);
            };
            if (j < S.NX) gx[j] = prof(S.NX);
            if (j < S.NY) gy[j] = prof(S.NY);
            if (j < S.NZ) gz[j] = prof(S.NZ);
        }
    }
}

__global__ void k_batch_image_add(BatchShot S, const float* __restrict__ slab, int fnx, int fny,
                                  int ox, int oy, int oz, float* __restrict__ img) {
    const long long n = (long long)S.nx * S.ny * S.nz;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % S.nx);
        const int y = (int)((i / S.nx) % S.ny);
        const int z = (int)(i / ((long long)S.nx * S.ny));
        img[((long long)(z + oz) * fny + (y + oy)) * fnx + (x + ox)] +=
            slab[((long long)z * S.ny + y) * S.NX + x + S.nb];
    }
}

}  // namespace

int batch_blocks_per_sm(int radius) {
    int n = 0;
    if (radius == 4)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch<4>, 256, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch<8>, 256, 0);
    return n;
}

cudaError_t launch_batch(int radius, const BatchArgs& a, int grid, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(16, 16);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (radius == 4) return cudaLaunchKernelEx(&cfg, k_batch<4>, a);
    if (radius == 8) return cudaLaunchKernelEx(&cfg, k_batch<8>, a);
    return cudaErrorInvalidValue;
}

cudaError_t launch_batch_prep(const BatchShot& sh, const float* vel_full, int full_nx, int full_ny,
                              int ox, int oy, int oz, double dt, float* c, float* gx, float* gy,
                              float* gz, cudaStream_t s) {
    const long long N = (long long)sh.NX * sh.NY * sh.NZ;
    long long blocks = (N + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    k_batch_prep<<<(unsigned)blocks, 256, 0, s>>>(sh, vel_full, full_nx, full_ny, ox, oy, oz,
                                                   (float)(dt * dt), c, gx, gy, gz);
    return cudaGetLastError();
}

cudaError_t launch_batch_image_add(const BatchShot& sh, int full_nx, int full_ny, int ox, int oy,
                                   int oz, float* image_full, cudaStream_t s) {
    const long long n = (long long)sh.nx * sh.ny * sh.nz;
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    k_batch_image_add<<<(unsigned)blocks, 256, 0, s>>>(sh, sh.img, full_nx, full_ny, ox, oy, oz,
                                                       image_full);
    return cudaGetLastError();
}

}  // namespace rtm
