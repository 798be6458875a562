// High-order star-stencil leapfrog step with fused sponge, snapshot,
// imaging and gradient epilogues (the per-time-step stencil of the paper's
// solver, Sec. II).
//
// 2.5D blocking: a thread block owns a TX x TY tile of x-y columns and marches
// through a slab of z planes. Each thread owns 4 consecutive x points of one
// row (one 16-byte vector). The current z plane of the tile, with an r-wide
// halo in x and y, is staged in shared memory (double buffered, one barrier
// per plane); the 2r+1 values of each thread's own column along z live in a
// register queue. Plane z+1 (queue head, halos, u^{n-1}, c and the epilogue
// operands) is loaded into registers while plane z is computed. x is the
// contiguous axis, the loop order the paper settles on (Sec. III).
//
// DRAM traffic per point: u^n, u^{n-1}, c read, u^{n+1} written (16 B);
// the halo re-reads of u^n come from L2, because all tiles of a z slab
// advance through z together.

#include "rtm_internal.h"
#include "stencil_common.cuh"

namespace rtm {

namespace {

template <int R, int MODE>
__global__ void __launch_bounds__(256, R == 4 ? 2 : 1) k_stencil(const __grid_constant__ StepArgs A) {
    using T = Tile<R>;
    __shared__ __align__(16) float sm[2][T::SH][T::SW];

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x0 = A.xorg + blockIdx.x * T::TX, y0 = A.yorg + blockIdx.y * T::TY;
    const int x = x0 + 4 * tx;
    const int y = y0 + ty;
    const int zb = A.zorg + blockIdx.z * A.zchunk;
    const int ze = min(A.zend, zb + A.zchunk);
    const bool xin = x < A.NX;  // NX % 4 == 0: a vector is all in or all out
    const bool yin = y < A.NY;
    const bool own = xin && yin;
    const size_t plane = (size_t)A.NX * (size_t)A.NY;
    const size_t col = (size_t)y * A.NX + x;

    // halo roles (fixed per thread)
    const bool hx_left = tx < T::HX;
    const bool hx_right = tx >= T::BX - T::HX;
    const int hx_x = hx_left ? (x0 - R + 4 * tx) : (x0 + T::TX + 4 * (tx - (T::BX - T::HX)));
    const bool hx_ok = (hx_left || hx_right) && yin && hx_x >= 0 && hx_x < A.NX;
    const size_t hx_col = (size_t)y * A.NX + (hx_ok ? hx_x : 0);
    const int hx_sc = hx_left ? 4 * tx : (R + T::TX + 4 * (tx - (T::BX - T::HX)));

    const bool hy_top = ty < R;
    const bool hy_bot = ty >= T::TY - R;
    const int hy_y = hy_top ? (y0 - R + ty) : (y0 + R + ty);
    const bool hy_ok = (hy_top || hy_bot) && xin && hy_y >= 0 && hy_y < A.NY;
    const size_t hy_col = (size_t)(hy_ok ? hy_y : 0) * A.NX + x;
    const int hy_sr = hy_top ? ty : ty + 2 * R;

    // model-region predicates for the slab epilogues
    const bool xm = (x + 3 >= A.nb) && (x < A.nb + A.nx);
    const bool ym = (y >= A.nb) && (y < A.nb + A.ny);
    const size_t slab_col = (size_t)(y - A.nb) * A.NX + x;
    const size_t slab_plane = (size_t)A.ny * A.NX;
    // reverse mode: all of this thread's cells lie in the model's x-y range
    const bool model_col = x >= A.nb && x + 3 < A.nb + A.nx && y >= A.nb && y < A.nb + A.ny;

    // sponge factor of the column, gz per plane
    F4 gxy = zero4();
    if (own) {
        const float gyv = A.gy[y];
#pragma unroll
        for (int i = 0; i < 4; i++) gxy.v[i] = A.gx[x + i] * gyv;
    }

    // register queue along z: q[i] = u(z - R + i)
    F4 q[2 * R + 1];
#pragma unroll
    for (int i = 0; i < 2 * R + 1; i++) {
        const int zz = zb - R + i;
        q[i] = (own && zz >= 0 && zz < A.NZ) ? ld_keep(A.u_cur + (size_t)zz * plane + col)
                                             : zero4();
    }
    // current-plane operands
    F4 hxv = hx_ok ? ld_keep(A.u_cur + (size_t)zb * plane + hx_col) : zero4();
    F4 hyv = hy_ok ? ld_keep(A.u_cur + (size_t)zb * plane + hy_col) : zero4();
    F4 up = own ? ld_stream(A.u_prev + (size_t)zb * plane + col) : zero4();
    F4 cc = own ? ld_stream(A.c + (size_t)zb * plane + col) : zero4();
    F4 e1 = zero4(), e2 = zero4();  // epilogue operands (snapshot, accumulator)
    auto load_epi = [&](int z, F4& s1, F4& s2) {
        if constexpr (MODE == MODE_BWD_IMAGE) {
            if (own && xm && ym && z >= A.nb && z < A.nb + A.nz) {
                const size_t o = (size_t)(z - A.nb) * slab_plane + slab_col;
                s1 = ld_stream(A.snap + (A.snap_padded ? (size_t)z * plane + col : o));
                s2 = ld_stream(A.acc + o);
            }
        } else if constexpr (MODE == MODE_BWD_GRAD) {
            if (own) {
                const size_t o = (size_t)z * plane + col;
                s1 = ld_stream(A.snap + o);
                s2 = ld_stream(A.acc + o);
            }
        }
    };
    load_epi(zb, e1, e2);

    float ssq = 0.f;  // MODE_FWD_SUMSQ: this thread's share of the sum of squares
    for (int z = zb; z < ze; z++) {
        float(*S)[T::SW] = sm[(z - zb) & 1];
        // stage plane z
        sts4(&S[R + ty][R + 4 * tx], q[R]);
        if (hx_left || hx_right) sts4(&S[R + ty][hx_sc], hxv);
        if (hy_top || hy_bot) sts4(&S[hy_sr][R + 4 * tx], hyv);

        // prefetch plane z + 1
        const int zn = z + 1;
        F4 qn = zero4(), hxn = zero4(), hyn = zero4(), upn = zero4(), ccn = zero4();
        F4 e1n = zero4(), e2n = zero4();
        if (zn < ze) {
            const int zq = zn + R;
            if (own && zq < A.NZ) qn = ld_keep(A.u_cur + (size_t)zq * plane + col);
            if (hx_ok) hxn = ld_keep(A.u_cur + (size_t)zn * plane + hx_col);
            if (hy_ok) hyn = ld_keep(A.u_cur + (size_t)zn * plane + hy_col);
            if (own) {
                upn = ld_stream(A.u_prev + (size_t)zn * plane + col);
                ccn = ld_stream(A.c + (size_t)zn * plane + col);
            }
            load_epi(zn, e1n, e2n);
        }
        __syncthreads();

        if (own) {
            // x neighbours: v[j] = u(x - R + j), j in [0, 4 + 2R)
            float v[4 + 2 * R];
#pragma unroll
            for (int h = 0; h < T::HX; h++) {
                const F4 l = lds4(&S[R + ty][4 * tx + 4 * h]);
                const F4 r = lds4(&S[R + ty][R + 4 * tx + 4 + 4 * h]);
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    v[4 * h + i] = l.v[i];
                    v[R + 4 + 4 * h + i] = r.v[i];
                }
            }
#pragma unroll
            for (int i = 0; i < 4; i++) v[R + i] = q[R].v[i];

            F4 lap;
#pragma unroll
            for (int i = 0; i < 4; i++) lap.v[i] = A.a[0] * q[R].v[i];
#pragma unroll
            for (int k = 1; k <= R; k++) {
                const F4 ym_ = lds4(&S[R + ty - k][R + 4 * tx]);
                const F4 yp_ = lds4(&S[R + ty + k][R + 4 * tx]);
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    const float px = v[R + i - k] + v[R + i + k];
                    const float py = ym_.v[i] + yp_.v[i];
                    const float pz = q[R - k].v[i] + q[R + k].v[i];
                    lap.v[i] = fmaf(A.a[k], (px + py) + pz, lap.v[i]);
                }
            }
            F4 out;
            if constexpr (MODE == MODE_REV) {
                // the sponge factor is 1 in the model region: the forward
                // update with the two time levels swapped
#pragma unroll
                for (int i = 0; i < 4; i++) out.v[i] = fmaf(cc.v[i], lap.v[i], 2.0f * q[R].v[i]) - up.v[i];
                if (!model_col) {  // cells outside the model keep their value
#pragma unroll
                    for (int i = 0; i < 4; i++) {
                        const int mx = x + i - A.nb, my = y - A.nb;
                        if (mx < 0 || mx >= A.nx || my < 0 || my >= A.ny) out.v[i] = up.v[i];
                    }
                }
            } else {
                const float gzv = A.gz[z];
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    const float g = gxy.v[i] * gzv;
                    out.v[i] = g * fmaf(cc.v[i], lap.v[i], 2.0f * q[R].v[i]) - (g * g) * up.v[i];
                }
            }
            const size_t o = (size_t)z * plane + col;
            st_stream(A.u_prev + o, out);

            if constexpr (MODE == MODE_FWD_SUMSQ) {
                if (ym && z >= A.nb && z < A.nb + A.nz) {
#pragma unroll
                    for (int i = 0; i < 4; i++)
                        if (x + i >= A.nb && x + i < A.nb + A.nx) ssq = fmaf(out.v[i], out.v[i], ssq);
                }
            } else if constexpr (MODE == MODE_FWD_SNAP) {
                if (xm && ym && z >= A.nb && z < A.nb + A.nz)
                    st_stream(A.snap + (size_t)(z - A.nb) * slab_plane + slab_col, out);
            } else if constexpr (MODE == MODE_BWD_IMAGE) {
                if (xm && ym && z >= A.nb && z < A.nb + A.nz) {
                    F4 acc;
#pragma unroll
                    for (int i = 0; i < 4; i++) acc.v[i] = fmaf(e1.v[i], out.v[i], e2.v[i]);
                    st_stream(A.acc + (size_t)(z - A.nb) * slab_plane + slab_col, acc);
                }
            } else if constexpr (MODE == MODE_FWD_LU) {
                st_stream(A.snap + o, lap);
            } else if constexpr (MODE == MODE_BWD_GRAD) {
                F4 acc;
#pragma unroll
                for (int i = 0; i < 4; i++) acc.v[i] = fmaf(out.v[i], e1.v[i], e2.v[i]);
                st_stream(A.acc + o, acc);
            }
        }

        // rotate
#pragma unroll
        for (int i = 0; i < 2 * R; i++) q[i] = q[i + 1];
        q[2 * R] = qn;
        hxv = hxn;
        hyv = hyn;
        up = upn;
        cc = ccn;
        e1 = e1n;
        e2 = e2n;
    }
    if constexpr (MODE == MODE_FWD_SUMSQ) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ssq += __shfl_xor_sync(0xffffffffu, ssq, o);
        if (((ty * T::BX + tx) & 31) == 0 && ssq != 0.f) atomicAdd(A.sumsq, (double)ssq);
    }
}

template <int R, int MODE>
cudaError_t launch_t(const StepArgs& a, cudaStream_t s) {
    using T = Tile<R>;
    dim3 block(T::BX, T::BY);
    dim3 grid((a.xend - a.xorg + T::TX - 1) / T::TX, (a.yend - a.yorg + T::TY - 1) / T::TY,
              (a.zend - a.zorg + a.zchunk - 1) / a.zchunk);
    if (a.xorg % 4 || a.xend <= a.xorg || a.yend <= a.yorg || a.zend <= a.zorg)
        return cudaErrorInvalidValue;
    k_stencil<R, MODE><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

template <int R>
cudaError_t launch_r(int mode, const StepArgs& a, cudaStream_t s) {
    switch (mode) {
        case MODE_FWD: return launch_t<R, MODE_FWD>(a, s);
        case MODE_FWD_SNAP: return launch_t<R, MODE_FWD_SNAP>(a, s);
        case MODE_BWD_IMAGE: return launch_t<R, MODE_BWD_IMAGE>(a, s);
        case MODE_FWD_LU: return launch_t<R, MODE_FWD_LU>(a, s);
        case MODE_BWD_GRAD: return launch_t<R, MODE_BWD_GRAD>(a, s);
        case MODE_REV: return launch_t<R, MODE_REV>(a, s);
        case MODE_FWD_SUMSQ: return launch_t<R, MODE_FWD_SUMSQ>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

int auto_zchunk(int radius, int NX, int NY, int NZ) {
    // aim for about four thread blocks per SM slot (152 SMs x 2 resident)
    const int tiles = ((NX + 63) / 64) * ((NY + 15) / 16);
    const int target = 152 * 2 * 4;
    int nzc = (target + tiles - 1) / tiles;
    if (nzc < 1) nzc = 1;
    int zc = (NZ + nzc - 1) / nzc;
    const int min_zc = 4 * radius;  // keep the 2r-plane queue warm-up small
    if (zc < min_zc) zc = min_zc;
    if (zc > NZ) zc = NZ;
    return zc < 1 ? 1 : zc;
}

cudaError_t launch_stencil(int radius, int mode, const StepArgs& a, cudaStream_t s) {
    if (a.zchunk < 1) return cudaErrorInvalidValue;
    switch (radius) {
        case 4: return launch_r<4>(mode, a, s);
        case 8: return launch_r<8>(mode, a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rtm
