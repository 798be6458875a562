// Small kernels around the stencil: model preparation, sponge profiles, the
// Ricker wavelet, source injection / receiver gather, adjoint injection,
// image and gradient finalisation, and the data misfit.

#include <math.h>

#include <algorithm>

#include "band.cuh"
#include "rtm_internal.h"

namespace rtm {

namespace {

constexpr int kStatusInvalid = 1;  // == RTM_ERR_INVALID

__device__ __forceinline__ void flag(int* status, int code) {
    if (status) atomicCAS(status, 0, code);
}

// padded linear index of model coordinates (x, y, z), or -1 if outside the
// padded grid
__device__ __forceinline__ long long rec_index(const Geometry& G, const int32_t* rec, int j) {
    const int x = rec[3 * j + 0] + G.nb, y = rec[3 * j + 1] + G.nb, z = rec[3 * j + 2] + G.nb;
    if (x < 0 || x >= G.NX || y < 0 || y >= G.NY || z < 0 || z >= G.NZ) return -1;
    return ((long long)z * G.NY + y) * G.NX + x;
}


// Cerjan-type profile: exp(-(0.015 (nb - d))^2) within nb cells of a face
__device__ __forceinline__ float sponge_1d(int i, int n, int nb) {
    const int d = min(i, n - 1 - i);
    if (d >= nb) return 1.0f;
    const double s = 0.015 * (double)(nb - d);
    return (float)exp(-s * s);
}

__global__ void k_sponge(Geometry G, float* gx, float* gy, float* gz) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < G.NX) gx[i] = sponge_1d(i, G.NX, G.nb);
    if (i < G.NY) gy[i] = sponge_1d(i, G.NY, G.nb);
    if (i < G.NZ) gz[i] = sponge_1d(i, G.NZ, G.nb);
}

// Ricker: w(t) = (1 - 2 pi^2 f0^2 (t - t0)^2) exp(-pi^2 f0^2 (t - t0)^2), in double
__global__ void k_wavelet(int nt, double dt, double f0, double t0, float* w) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nt) return;
    const double pf = 3.14159265358979323846 * f0 * ((double)n * dt - t0);
    const double a = pf * pf;
    w[n] = (float)((1.0 - 2.0 * a) * exp(-a));
}

// c = v^2 dt^2 on the padded grid (edge padding); max v^2 and validity over
// the model cells
__global__ void k_model_prep(Geometry G, const float* __restrict__ vel, int squared, float dt2,
                             float* __restrict__ c, unsigned int* vmax_bits, int* bad) {
    const long long N = (long long)G.NX * G.NY * G.NZ;
    const long long stride = (long long)gridDim.x * blockDim.x;
    float local_max = 0.0f;
    int local_bad = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        const long long plane = (long long)G.NX * G.NY;
        const int z = (int)(i / plane);
        const int y = (int)((i % plane) / G.NX);
        const int x = (int)(i % G.NX);
        const int mx = min(max(x - G.nb, 0), G.nx - 1);
        const int my = min(max(y - G.nb, 0), G.ny - 1);
        const int mz = min(max(z - G.nb, 0), G.nz - 1);
        const float v = vel[((long long)mz * G.ny + my) * G.nx + mx];
        const float v2 = squared ? v : v * v;
        c[i] = v2 * dt2;
        const bool interior = (x - G.nb == mx) && (y - G.nb == my) && (z - G.nb == mz);
        if (interior) {
            if (!(isfinite(v) && v > 0.0f)) local_bad = 1;
            else local_max = fmaxf(local_max, v2);
        }
    }
    // warp reduction then one atomic per warp
    for (int o = 16; o > 0; o >>= 1) {
        local_max = fmaxf(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
        local_bad |= __shfl_xor_sync(0xffffffffu, local_bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(vmax_bits, __float_as_uint(local_max));  // non-negative floats order as uints
        if (local_bad) atomicOr(bad, 1);
    }
}

__global__ void k_fwd_aux(Geometry G, const float* __restrict__ u_cur, float* u_prev,
                          const float* __restrict__ c, const float* gx, const float* gy,
                          const float* gz, const int32_t* __restrict__ rec, int nrec,
                          float* data_row, long long src, const float* w_n, float inv_dx3,
                          int* status) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < nrec) {
        if (data_row) {
            const long long i = rec_index(G, rec, j);
            if (i < 0) flag(status, kStatusInvalid);
            data_row[j] = i >= 0 ? u_cur[i] : 0.0f;
        }
    } else if (j == nrec && w_n) {
        // the stencil computes g(...) - g^2 u_prev: lowering u_prev[s] by
        // c_s w / (dx^3 g_s^2) adds c_s w / dx^3 to u^{n+1}[s]
        const float g = sponge_at(G, gx, gy, gz, src);
        u_prev[src] -= c[src] * (*w_n) * inv_dx3 / (g * g);
    }
}

__global__ void k_bwd_aux(Geometry G, const float* __restrict__ mu_cur, float* mu_prev,
                          const float* __restrict__ c, const float* gx, const float* gy,
                          const float* gz, const int32_t* __restrict__ rec, int nrec,
                          const float* __restrict__ r_row, long long src, float* src_adj_slot,
                          float* grad_acc, const float* w_n, float inv_dx3, int* status) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < nrec) {
        if (r_row) {
            const long long i = rec_index(G, rec, j);
            if (i < 0) {
                flag(status, kStatusInvalid);
            } else {
                // lowering mu_prev[i] by c r / (dx^3 g) adds c g r / dx^3 to mu^m[i]
                const float g = sponge_at(G, gx, gy, gz, i);
                atomicAdd(&mu_prev[i], -c[i] * r_row[j] * inv_dx3 / g);
            }
        }
    } else if (j == nrec) {
        const float g = sponge_at(G, gx, gy, gz, src);
        const float m = mu_cur[src];
        if (src_adj_slot) *src_adj_slot = m / g;
        if (grad_acc && w_n) grad_acc[src] += m * (*w_n) * inv_dx3 / g;
    }
}

__global__ void k_image_finalize(Geometry G, const float* __restrict__ slab,
                                 float* __restrict__ image) {
    const long long n = (long long)G.nx * G.ny * G.nz;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const long long zy = i / G.nx;
        const int x = (int)(i % G.nx);
        image[i] += slab[zy * G.NX + x + G.nb];
    }
}

// source illumination: illum[z][y][x] += u^2 of the model columns of a
// snapshot slab [nz][ny][NX]; 16-byte vectors along x when both rows allow
// boundary band of the model region: gather from a padded field / scatter into it
__global__ void k_band_copy(Geometry G, int r, float* __restrict__ field,
                            float* __restrict__ band, long long n, int to_field) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < n; b += stride) {
        int mx, my, mz;
        band_cell(b, G.nx, G.ny, G.nz, r, mx, my, mz);
        const long long i =
            ((long long)(mz + G.nb) * G.NY + (my + G.nb)) * G.NX + (mx + G.nb);
        if (to_field)
            field[i] = band[b];
        else
            band[b] = field[i];
    }
}

// first element of model row zy = z ny + y: in the slab, or in a padded field
__device__ __forceinline__ long long model_row(const Geometry& G, long long zy, int padded) {
    if (!padded) return zy * G.NX + G.nb;
    const long long z = zy / G.ny;
    return ((z + G.nb) * G.NY + (zy - z * G.ny) + G.nb) * G.NX + G.nb;
}

__global__ void k_illum_add(Geometry G, const float* __restrict__ slab,
                            float* __restrict__ illum, int vec, int padded) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    if (vec) {
        const int nx4 = G.nx >> 2;
        const long long n4 = (long long)nx4 * G.ny * G.nz;
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
            const long long zy = i / nx4;
            const int x4 = (int)(i - zy * nx4);
            const float4 u =
                __ldcs(reinterpret_cast<const float4*>(slab + model_row(G, zy, padded)) + x4);
            float4* d = reinterpret_cast<float4*>(illum + zy * G.nx) + x4;
            float4 a = *d;
            a.x = fmaf(u.x, u.x, a.x);
            a.y = fmaf(u.y, u.y, a.y);
            a.z = fmaf(u.z, u.z, a.z);
            a.w = fmaf(u.w, u.w, a.w);
            *d = a;
        }
        return;
    }
    const long long n = (long long)G.nx * G.ny * G.nz;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const long long zy = i / G.nx;
        const int x = (int)(i % G.nx);
        const float u = slab[model_row(G, zy, padded) + x];
        illum[i] = fmaf(u, u, illum[i]);
    }
}

// largest value of a non-negative array (float bits compare as unsigned)
__global__ void k_max_nonneg(const float* __restrict__ a, long long n, unsigned int* bits) {
    float m = 0.f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        m = fmaxf(m, a[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(bits, __float_as_uint(m));
}

// out = image / (illum + eps_rel * max illum)
__global__ void k_image_normalize(const float* __restrict__ image, const float* __restrict__ illum,
                                  long long n, const unsigned int* max_bits, float eps_rel,
                                  float* __restrict__ out) {
    const float floor_ = eps_rel * __uint_as_float(*max_bits);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = image[i] / (illum[i] + floor_);
}

// out = -L image on the model grid, zero outside it; a[0] = 3 a0 / dx^2,
// a[k] = a_k / dx^2
__global__ void k_image_laplacian(const float* __restrict__ image, int nx, int ny, int nz,
                                  LapWeights w, float* __restrict__ out) {
    const long long n = (long long)nx * ny * nz;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long sy = nx, sz = (long long)nx * ny;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / sz);
        float acc = w.a[0] * image[i];
        for (int k = 1; k <= w.r; k++) {
            float s = 0.f;
            if (x + k < nx) s += image[i + k];
            if (x - k >= 0) s += image[i - k];
            if (y + k < ny) s += image[i + k * sy];
            if (y - k >= 0) s += image[i - k * sy];
            if (z + k < nz) s += image[i + k * sz];
            if (z - k >= 0) s += image[i - k * sz];
            acc = fmaf(w.a[k], s, acc);
        }
        out[i] = -acc;
    }
}

__device__ __forceinline__ void fold_range(int m, int n, int nb, int N, int& lo, int& hi) {
    lo = (m == 0) ? 0 : m + nb;
    hi = (m == n - 1) ? N - 1 : m + nb;
}

// grad_v2[model cell] = dt^2 * sum over the padded cells copied from that
// cell of dx^3 acc / c (the transpose of the edge padding)
__global__ void k_grad_finalize(Geometry G, const float* __restrict__ acc,
                                const float* __restrict__ c, double dx3, double dt2,
                                float* __restrict__ grad) {
    const long long n = (long long)G.nx * G.ny * G.nz;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int x = (int)(i % G.nx);
        const int y = (int)((i / G.nx) % G.ny);
        const int z = (int)(i / ((long long)G.nx * G.ny));
        int x0, x1, y0, y1, z0, z1;
        fold_range(x, G.nx, G.nb, G.NX, x0, x1);
        fold_range(y, G.ny, G.nb, G.NY, y0, y1);
        fold_range(z, G.nz, G.nb, G.NZ, z0, z1);
        double s = 0.0;
        for (int zz = z0; zz <= z1; zz++)
            for (int yy = y0; yy <= y1; yy++)
                for (int xx = x0; xx <= x1; xx++) {
                    const long long p = ((long long)zz * G.NY + yy) * G.NX + xx;
                    s += (double)acc[p] / (double)c[p];
                }
        grad[i] = (float)(s * dx3 * dt2);
    }
}

__global__ void k_misfit(const float* __restrict__ d, const float* __restrict__ obs, long long n,
                         float* resid, double* J) {
    double local = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float r = d[i] - obs[i];
        if (resid) resid[i] = r;
        local += 0.5 * (double)r * (double)r;
    }
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    __shared__ double warp_sum[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) warp_sum[wid] = local;
    __syncthreads();
    if (wid == 0) {
        double v = lane < (int)(blockDim.x >> 5) ? warp_sum[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) atomicAdd(J, v);
    }
}

// any non-finite value among n floats sets the status word to
// RTM_ERR_NUMERIC (6); 16-byte loads when the base is aligned
__global__ void k_finite_scan(const float* __restrict__ f, long long n, int vec, int* status) {
    bool bad = false;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (vec) {
        const long long n4 = n / 4;
        const float4* f4 = reinterpret_cast<const float4*>(f);
        for (long long i = t; i < n4; i += stride) {
            const float4 v = __ldcs(f4 + i);
            bad |= !isfinite(v.x) || !isfinite(v.y) || !isfinite(v.z) || !isfinite(v.w);
        }
        for (long long i = 4 * n4 + t; i < n; i += stride) bad |= !isfinite(f[i]);
    } else {
        for (long long i = t; i < n; i += stride) bad |= !isfinite(__ldcs(f + i));
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) flag(status, 6);
}

// decimated storage, coding: keep every other sample of the model region
// on each axis, coarse[kz][ky][kx] = u[nb + 2 kz][nb + 2 ky][nb + 2 kx] of a
// padded field; coarse sides are (n + 1) / 2. A block walks coarse rows
// (ky, kz), its threads along x
__global__ void k_decimate(Geometry G, const float* __restrict__ u, float* __restrict__ coarse,
                           int cx, int cy, int cz) {
    for (int row = blockIdx.x; row < cy * cz; row += gridDim.x) {
        const int ky = row % cy, kz = row / cy;
        const float* src = u + ((long long)(G.nb + 2 * kz) * G.NY + (G.nb + 2 * ky)) * G.NX + G.nb;
        float* dst = coarse + (long long)row * cx;
        for (int kx = threadIdx.x; kx < cx; kx += blockDim.x) dst[kx] = __ldcs(src + 2 * kx);
    }
}

// per axis: fine sample j from coarse samples i0 and i0 + 1 with weight w1 on
// the second: an even sample is a kept one; an odd sample is the mean of its
// two neighbours, or a copy of the left one past the last kept sample
__device__ __forceinline__ void lin_axis(int j, int nc, int& i0, float& w1) {
    i0 = j >> 1;
    w1 = ((j & 1) && i0 + 1 < nc) ? 0.5f : 0.0f;
}

// decimated storage, decoding: linear interpolation along each axis back to
// the model region of a snapshot slab [nz][ny][NX] (columns nb .. nb + nx);
// the weights (1, 1/2) are exact. One warp per output row (y, z): each lane
// interpolates one kept column along y and z from the four coarse rows
// (coalesced loads), takes its right neighbour's value by a shuffle, and
// writes the even output sample (the kept column) and the odd one (the mean
// of the two, or a copy past the last kept column)
__global__ void k_upsample(Geometry G, const float* __restrict__ coarse, int cx, int cy, int cz,
                           float* __restrict__ slab) {
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    // rows start 16-byte aligned (NX % 4 == 0): output pairs are 8-byte
    // aligned when the model's first column is even
    const bool pairs = (G.nb % 2) == 0;
    for (long long row = warp; row < (long long)G.ny * G.nz; row += nwarps) {
        const int y = (int)(row % G.ny), z = (int)(row / G.ny);
        int y0, z0;
        float wy, wz;
        lin_axis(y, cy, y0, wy);
        lin_axis(z, cz, z0, wz);
        const int y1 = wy > 0.f ? y0 + 1 : y0, z1 = wz > 0.f ? z0 + 1 : z0;
        const float* r00 = coarse + ((long long)z0 * cy + y0) * cx;
        const float* r01 = coarse + ((long long)z0 * cy + y1) * cx;
        const float* r10 = coarse + ((long long)z1 * cy + y0) * cx;
        const float* r11 = coarse + ((long long)z1 * cy + y1) * cx;
        float* out = slab + row * G.NX + G.nb;
        auto kept = [&](int k) {  // kept column k interpolated along y, then z
            const float a0 = (1.f - wy) * __ldg(r00 + k) + wy * __ldg(r01 + k);
            const float a1 = (1.f - wy) * __ldg(r10 + k) + wy * __ldg(r11 + k);
            return (1.f - wz) * a0 + wz * a1;
        };
        // four groups of 32 kept columns at a time: their loads are in flight together
        constexpr int U = 4;
        for (int base = 0; base < cx; base += 32 * U) {
            float bk[U + 1];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int k = base + 32 * u + lane;
                bk[u] = k < cx ? kept(k) : 0.f;
            }
            const int kl = base + 32 * U;  // the column after the last group, for lane 31
            bk[U] = (lane == 31 && kl < cx) ? kept(kl) : 0.f;
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int k = base + 32 * u + lane;
                // the next kept column: lane + 1's, or for lane 31 the next
                // group's first (lane 0), or the extra column after the last group
                const float right = __shfl_down_sync(0xffffffffu, bk[u], 1);
                const float head = __shfl_sync(0xffffffffu, u + 1 < U ? bk[u + 1] : 0.f, 0);
                const float bn = lane < 31 ? right : (u + 1 < U ? head : bk[U]);
                if (k < cx) {
                    const float odd = k + 1 < cx ? 0.5f * bk[u] + 0.5f * bn : bk[u];
                    if (pairs && 2 * k + 1 < G.nx) {  // whole lines per warp
                        __stcs(reinterpret_cast<float2*>(out + 2 * k), make_float2(bk[u], odd));
                    } else {
                        __stcs(out + 2 * k, bk[u]);
                        if (2 * k + 1 < G.nx) __stcs(out + 2 * k + 1, odd);
                    }
                }
            }
        }
    }
}

int grid_for(long long n, int block) {
    long long g = (n + block - 1) / block;
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

cudaError_t launch_sponge(const Geometry& G, float* gx, float* gy, float* gz, cudaStream_t s) {
    const int n = max(G.NX, max(G.NY, G.NZ));
    k_sponge<<<(n + 255) / 256, 256, 0, s>>>(G, gx, gy, gz);
    return cudaGetLastError();
}

cudaError_t launch_wavelet(int nt, double dt, double f0, double t0, float* w, cudaStream_t s) {
    k_wavelet<<<(nt + 255) / 256, 256, 0, s>>>(nt, dt, f0, t0, w);
    return cudaGetLastError();
}

cudaError_t launch_model_prep(const Geometry& G, const float* vel, int squared, double dt,
                              float* c, unsigned int* vmax_bits, int* bad, cudaStream_t s) {
    const long long N = (long long)G.NX * G.NY * G.NZ;
    k_model_prep<<<grid_for(N, 256), 256, 0, s>>>(G, vel, squared, (float)(dt * dt), c,
                                                  vmax_bits, bad);
    return cudaGetLastError();
}

cudaError_t launch_fwd_aux(const Geometry& G, const float* u_cur, float* u_prev, const float* c,
                           const float* gx, const float* gy, const float* gz,
                           const int32_t* rec, int nrec, float* data_row, long long src,
                           const float* w_n, float inv_dx3, int* status, cudaStream_t s) {
    const int n = nrec + 1;
    k_fwd_aux<<<(n + 255) / 256, 256, 0, s>>>(G, u_cur, u_prev, c, gx, gy, gz, rec, nrec,
                                              data_row, src, w_n, inv_dx3, status);
    return cudaGetLastError();
}

cudaError_t launch_bwd_aux(const Geometry& G, const float* mu_cur, float* mu_prev,
                           const float* c, const float* gx, const float* gy, const float* gz,
                           const int32_t* rec, int nrec, const float* r_row, long long src,
                           float* src_adj_slot, float* grad_acc, const float* w_n,
                           float inv_dx3, int* status, cudaStream_t s) {
    const int n = nrec + 1;
    k_bwd_aux<<<(n + 255) / 256, 256, 0, s>>>(G, mu_cur, mu_prev, c, gx, gy, gz, rec, nrec,
                                              r_row, src, src_adj_slot, grad_acc, w_n,
                                              inv_dx3, status);
    return cudaGetLastError();
}

cudaError_t launch_image_finalize(const Geometry& G, const float* slab, float* image,
                                  cudaStream_t s) {
    const long long n = (long long)G.nx * G.ny * G.nz;
    k_image_finalize<<<grid_for(n, 256), 256, 0, s>>>(G, slab, image);
    return cudaGetLastError();
}

cudaError_t launch_band_copy(const Geometry& G, int r, float* field, float* band, int to_field,
                             cudaStream_t s) {
    const long long n = band_cells(G.nx, G.ny, G.nz, r);
    if (n <= 0) return cudaSuccess;
    k_band_copy<<<grid_for(n, 256), 256, 0, s>>>(G, r, field, band, n, to_field);
    return cudaGetLastError();
}

cudaError_t launch_illum_add(const Geometry& G, const float* slab, float* illum, int padded,
                             cudaStream_t s) {
    const long long n = (long long)G.nx * G.ny * G.nz;
    // slab and padded rows start 16-byte aligned (NX % 4 == 0); the model
    // columns do when nb % 4 == 0, the illumination rows when nx % 4 == 0
    const int vec = (G.nb % 4 == 0) && (G.nx % 4 == 0) &&
                    (reinterpret_cast<uintptr_t>(illum) % 16 == 0) &&
                    (reinterpret_cast<uintptr_t>(slab) % 16 == 0);
    k_illum_add<<<grid_for(vec ? n / 4 : n, 256), 256, 0, s>>>(G, slab, illum, vec, padded);
    return cudaGetLastError();
}

cudaError_t launch_image_normalize(const float* image, const float* illum, long long n,
                                   unsigned int* max_bits, float eps_rel, float* out,
                                   cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(max_bits, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    k_max_nonneg<<<grid_for(n, 256), 256, 0, s>>>(illum, n, max_bits);
    k_image_normalize<<<grid_for(n, 256), 256, 0, s>>>(image, illum, n, max_bits, eps_rel, out);
    return cudaGetLastError();
}

cudaError_t launch_image_laplacian(const float* image, int nx, int ny, int nz,
                                   const LapWeights& w, float* out, cudaStream_t s) {
    const long long n = (long long)nx * ny * nz;
    k_image_laplacian<<<grid_for(n, 256), 256, 0, s>>>(image, nx, ny, nz, w, out);
    return cudaGetLastError();
}

cudaError_t launch_grad_finalize(const Geometry& G, const float* acc, const float* c,
                                 double dx3, double dt2, float* grad_v2, cudaStream_t s) {
    const long long n = (long long)G.nx * G.ny * G.nz;
    k_grad_finalize<<<grid_for(n, 256), 256, 0, s>>>(G, acc, c, dx3, dt2, grad_v2);
    return cudaGetLastError();
}

cudaError_t launch_finite_scan(const float* f, long long n, int* status, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int vec = reinterpret_cast<uintptr_t>(f) % 16 == 0;
    k_finite_scan<<<grid_for(vec ? n / 4 + 1 : n, 256), 256, 0, s>>>(f, n, vec, status);
    return cudaGetLastError();
}

// rows of a row-walking kernel: 16 resident blocks per SM on 152 SMs at most
static int row_blocks(long long rows) { return (int)(rows < 152 * 16 ? rows : 152 * 16); }

cudaError_t launch_decimate(const Geometry& G, const float* u, float* coarse, cudaStream_t s) {
    const int cx = (G.nx + 1) / 2, cy = (G.ny + 1) / 2, cz = (G.nz + 1) / 2;
    const int tb = cx > 128 ? 256 : 128;
    k_decimate<<<row_blocks((long long)cy * cz), tb, 0, s>>>(G, u, coarse, cx, cy, cz);
    return cudaGetLastError();
}

cudaError_t launch_upsample(const Geometry& G, const float* coarse, float* slab, cudaStream_t s) {
    const int cx = (G.nx + 1) / 2, cy = (G.ny + 1) / 2, cz = (G.nz + 1) / 2;
    // a warp per row: 256-thread blocks, eight resident per SM
    const long long rows = (long long)G.ny * G.nz;
    const int blocks = (int)std::min<long long>((rows + 7) / 8, 152 * 8);
    k_upsample<<<blocks, 256, 0, s>>>(G, coarse, cx, cy, cz, slab);
    return cudaGetLastError();
}

cudaError_t launch_misfit(const float* d, const float* obs, long long n, float* resid, double* J,
                          cudaStream_t s) {
    k_misfit<<<grid_for(n, 256), 256, 0, s>>>(d, obs, n, resid, J);
    return cudaGetLastError();
}

}  // namespace rtm
