// Off-grid sources and receivers: Kaiser-windowed sinc tap tables (Hicks
// 2002) and the source / receiver kernels that use them.
//
// The paper's time step includes "interpolation where necessary" (Sec. II).
// A point between grid points is spread over its 8 nearest grid points per
// axis with the weights sinc(i - xi) I0(b sqrt(1 - ((i - xi) / R)^2)) / I0(b)
// (R = 4, b = 4.14); on an axis where it sits on a grid point, over that
// point alone with weight 1, so an on-grid point gives exactly the on-grid
// kernels' results. The weights are computed on the host in double
// precision: I0 by its power series, sinc through the sine of the distance
// to the nearest integer (exactly zero at the other grid points).

#include <math.h>
#include <string.h>

#include "../../include/rtm.h"
#include "rtm_internal.h"

namespace rtm {

namespace {

constexpr int kHalfWidth = 4;
constexpr double kKaiserB = 4.14;
constexpr double kPi = 3.14159265358979323846;

// modified Bessel function of the first kind, order 0: sum_k ((x/2)^k / k!)^2
double bessel_i0(double x) {
    const double q = 0.25 * x * x;
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 200; k++) {
        term *= q / ((double)k * k);
        sum += term;
        if (term < 1e-17 * sum) break;
    }
    return sum;
}

// sin(pi d) / (pi d), exactly 0 at nonzero integers and 1 at 0
double sinc(double d) {
    if (d == 0.0) return 1.0;
    const double n = nearbyint(d);
    const double f = d - n;
    const double s = sin(kPi * f) * ((((long long)n) & 1) ? -1.0 : 1.0);
    return s / (kPi * d);
}

// taps of one axis inside [0, n): first index and weights; false if xi is
// outside the grid
bool axis_taps(double xi, int n, int32_t* first, int32_t* count, float* w) {
    if (!(xi >= 0.0) || !(xi <= (double)(n - 1))) return false;
    if (xi == floor(xi)) {
        *first = (int32_t)xi;
        *count = 1;
        w[0] = 1.0f;
        for (int k = 1; k < 8; k++) w[k] = 0.0f;
        return true;
    }
    const int lo = (int)floor(xi) - kHalfWidth + 1;
    const double i0b = bessel_i0(kKaiserB);
    int a = lo, b = lo + 2 * kHalfWidth;  // [a, b) inside the grid
    if (a < 0) a = 0;
    if (b > n) b = n;
    *first = a;
    *count = b - a;
    for (int k = 0; k < 8; k++) w[k] = 0.0f;
    for (int i = a; i < b; i++) {
        const double d = (double)i - xi;
        const double r = d / kHalfWidth;
        const double win = bessel_i0(kKaiserB * sqrt(fmax(0.0, 1.0 - r * r))) / i0b;
        w[i - a] = (float)(sinc(d) * win);
    }
    return true;
}

// tap t of a point: padded linear index (or -1 outside the grid) and weight
__device__ __forceinline__ long long tap_of(const Geometry& G, const rtm_point_taps& P, int t,
                                            float* weight) {
    const int a = t % P.nx, b = (t / P.nx) % P.ny, c = t / (P.nx * P.ny);
    const int x = P.i0 + a, y = P.j0 + b, z = P.k0 + c;
    *weight = P.wx[a] * P.wy[b] * P.wz[c];
    if (x < 0 || x >= G.NX || y < 0 || y >= G.NY || z < 0 || z >= G.NZ) return -1;
    return ((long long)z * G.NY + y) * G.NX + x;
}

__device__ __forceinline__ int ntaps(const rtm_point_taps& P) {
    const bool ok = P.nx >= 1 && P.nx <= 8 && P.ny >= 1 && P.ny <= 8 && P.nz >= 1 && P.nz <= 8;
    return ok ? P.nx * P.ny * P.nz : 0;
}

__device__ __forceinline__ float warp_sum(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// one warp per point: warps 0 .. nrec - 1 gather d[n-1] = sum_t W_t u^n[t]
// (if data_row), warp nrec lowers u^{n-1} at the source taps by
// c W w / (dx^3 g^2) so that the stencil adds c W w / dx^3 to u^{n+1}
__global__ void k_fwd_aux_off(Geometry G, const float* __restrict__ u_cur, float* u_prev,
                              const float* __restrict__ c, const float* gx, const float* gy,
                              const float* gz, const rtm_point_taps* __restrict__ taps, int nrec,
                              float* data_row, const float* w_n, float inv_dx3, int* status) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp < nrec) {
        if (!data_row) return;
        const rtm_point_taps P = taps[1 + warp];
        const int n = ntaps(P);
        if (n == 0 && lane == 0) atomicCAS(status, 0, RTM_ERR_INVALID);
        float acc = 0.f;
        for (int t = lane; t < n; t += 32) {
            float wt;
            const long long i = tap_of(G, P, t, &wt);
            if (i < 0) {
                atomicCAS(status, 0, RTM_ERR_INVALID);
                continue;
            }
            acc += wt * u_cur[i];
        }
        acc = warp_sum(acc);
        if (lane == 0) data_row[warp] = acc;
    } else if (warp == nrec && w_n) {
        const rtm_point_taps P = taps[0];
        const int n = ntaps(P);
        if (n == 0 && lane == 0) atomicCAS(status, 0, RTM_ERR_INVALID);
        for (int t = lane; t < n; t += 32) {
            float wt;
            const long long i = tap_of(G, P, t, &wt);
            if (i < 0) {
                atomicCAS(status, 0, RTM_ERR_INVALID);
                continue;
            }
            const float g = sponge_at(G, gx, gy, gz, i);
            u_prev[i] -= c[i] * (wt * (*w_n)) * inv_dx3 / (g * g);
        }
    }
}

// one warp per point: warps 0 .. nrec - 1 lower mu^{m-1} at the receiver taps
// by c W r / (dx^3 g) (overlapping taps of neighbouring receivers: atomics),
// warp nrec records the source trace sum_t W_t mu^m[t] / g_t (if requested)
__global__ void k_bwd_aux_off(Geometry G, const float* __restrict__ mu_cur, float* mu_prev,
                              const float* __restrict__ c, const float* gx, const float* gy,
                              const float* gz, const rtm_point_taps* __restrict__ taps, int nrec,
                              const float* __restrict__ r_row, float* src_adj_slot,
                              float inv_dx3, int* status) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp < nrec) {
        if (!r_row) return;
        const rtm_point_taps P = taps[1 + warp];
        const int n = ntaps(P);
        if (n == 0 && lane == 0) atomicCAS(status, 0, RTM_ERR_INVALID);
        const float r = r_row[warp];
        for (int t = lane; t < n; t += 32) {
            float wt;
            const long long i = tap_of(G, P, t, &wt);
            if (i < 0) {
                atomicCAS(status, 0, RTM_ERR_INVALID);
                continue;
            }
            const float g = sponge_at(G, gx, gy, gz, i);
            atomicAdd(&mu_prev[i], -c[i] * (wt * r) * inv_dx3 / g);
        }
    } else if (warp == nrec && src_adj_slot) {
        const rtm_point_taps P = taps[0];
        const int n = ntaps(P);
        float acc = 0.f;
        for (int t = lane; t < n; t += 32) {
            float wt;
            const long long i = tap_of(G, P, t, &wt);
            if (i >= 0) acc += (wt * mu_cur[i]) / sponge_at(G, gx, gy, gz, i);
        }
        acc = warp_sum(acc);
        if (lane == 0) *src_adj_slot = acc;
    }
}

}  // namespace

cudaError_t launch_fwd_aux_off(const Geometry& G, const float* u_cur, float* u_prev,
                               const float* c, const float* gx, const float* gy,
                               const float* gz, const rtm_point_taps* taps, int nrec,
                               float* data_row, const float* w_n, float inv_dx3, int* status,
                               cudaStream_t s) {
    const long long threads = 32LL * (nrec + 1);
    k_fwd_aux_off<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
        G, u_cur, u_prev, c, gx, gy, gz, taps, nrec, data_row, w_n, inv_dx3, status);
    return cudaGetLastError();
}

cudaError_t launch_bwd_aux_off(const Geometry& G, const float* mu_cur, float* mu_prev,
                               const float* c, const float* gx, const float* gy,
                               const float* gz, const rtm_point_taps* taps, int nrec,
                               const float* r_row, float* src_adj_slot, float inv_dx3,
                               int* status, cudaStream_t s) {
    const long long threads = 32LL * (nrec + 1);
    k_bwd_aux_off<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
        G, mu_cur, mu_prev, c, gx, gy, gz, taps, nrec, r_row, src_adj_slot, inv_dx3, status);
    return cudaGetLastError();
}

}  // namespace rtm

extern "C" size_t rtm_offgrid_taps(const rtm_params* p, const double* h_src_xyz, int32_t nrec,
                                   const double* h_rec_xyz, rtm_point_taps* h_out,
                                   size_t out_count) {
    if (rtm_validate(p) != RTM_OK) return 0;
    if (!h_src_xyz || nrec < 0 || (nrec > 0 && !h_rec_xyz)) {
        rtm::set_error(RTM_ERR_INVALID, "source or receiver positions are NULL");
        return 0;
    }
    const int NX = p->nx + 2 * p->nb, NY = p->ny + 2 * p->nb, NZ = p->nz + 2 * p->nb;
    const size_t n = 1 + (size_t)nrec;
    const bool write = h_out && out_count >= n;
    for (size_t k = 0; k < n; k++) {
        const double* xyz = k == 0 ? h_src_xyz : h_rec_xyz + 3 * (k - 1);
        rtm_point_taps P;
        memset(&P, 0, sizeof P);
        if (!rtm::axis_taps(xyz[0] + p->nb, NX, &P.i0, &P.nx, P.wx) ||
            !rtm::axis_taps(xyz[1] + p->nb, NY, &P.j0, &P.ny, P.wy) ||
            !rtm::axis_taps(xyz[2] + p->nb, NZ, &P.k0, &P.nz, P.wz)) {
            rtm::set_error(RTM_ERR_INVALID, "point %zu (%g, %g, %g) outside the padded grid", k,
                           xyz[0], xyz[1], xyz[2]);
            return 0;
        }
        if (write) h_out[k] = P;
    }
    return n;
}
