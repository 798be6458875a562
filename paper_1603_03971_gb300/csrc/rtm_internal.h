// Internal declarations shared by the translation units of librtm.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

struct rtm_point_taps;  // include/rtm.h

namespace rtm {

// Stencil kernel modes. All of them compute the same leapfrog update
//   out = g (2 u + c L u) - g^2 prev
// and differ only in what they do besides.
enum StencilMode : int {
    MODE_FWD = 0,       // plain step (forward, or backward without imaging)
    MODE_FWD_SNAP = 1,  // + write the new field on the model slab (imaging snapshot)
    MODE_BWD_IMAGE = 2, // + image slab += snapshot * new field
    MODE_FWD_LU = 3,    // + write L u on the padded grid (gradient snapshot)
    MODE_BWD_GRAD = 4,  // + grad += new field * snapshot (L u), padded grid
    // (5: the batched launch, in the statistics only)
    MODE_REV = 6,       // reverse step over the model region, sponge factor 1:
                        // u^{n-1} = 2u^n + c L u^n - u^{n+1} (cells outside the
                        // model keep their value)
    MODE_FWD_SUMSQ = 7, // + sum of squares of the new field over the model region (+= *sumsq)
    MODE_COUNT = 8
};

constexpr int kMaxRadius = 8;

// Centred 2r-order second-derivative weights (closed form, rtm_api.cu):
// a_k = 2 (-1)^(k+1) (r!)^2 / (k^2 (r-k)! (r+k)!), a_0 = -2 sum_k a_k.
void stencil_weights(int r, double* a);
// The stencil kernels' coefficients from those weights: a[0] = 3 a_0 / dx^2
// (the centre term of the three axes), a[k] = a_k / dx^2; a has r + 1 entries.
void step_weights(int r, double dx, float* a);

// Arguments of one stencil launch. The "slab" layout used by imaging
// snapshots and the internal image is [nz][ny][NX]: z and y restricted to the
// model region, x over the full padded row, so that it shares the 16-byte
// alignment of the padded fields.
struct StepArgs {
    const float* u_cur;  // u^n (read only)
    float* u_prev;       // in: u^{n-1}; out: u^{n+1} (updated in place)
    const float* c;      // v^2 dt^2
    const float* gx;     // sponge profiles
    const float* gy;
    const float* gz;
    float* snap;         // snapshot or band of one state (mode dependent)
    float* acc;          // image slab or gradient accumulator
    int NX, NY, NZ;      // padded grid
    int nb, nx, ny, nz;  // model region
    int zchunk;          // z planes per thread block
    // region the launch covers: x in [xorg, xend) (xorg % 4 == 0), y in
    // [yorg, yend), z in [zorg, zend); the whole padded grid except for
    // MODE_REV, which covers the model region
    int xorg, xend, yorg, yend, zorg, zend;
    int snap_padded;     // MODE_BWD_IMAGE: snapshot on the padded grid instead of the slab
    double* sumsq;       // MODE_FWD_SUMSQ: accumulator of the model region's sum of squares
    float a[kMaxRadius + 1];  // a[0] = 3 a0 / dx^2, a[k] = a_k / dx^2
};

// the region of a mode: the padded grid, or the model region for MODE_REV
inline void set_region(StepArgs& a, int mode) {
    if (mode == MODE_REV) {
        a.xorg = a.nb & ~3;
        a.xend = a.nb + a.nx;
        a.yorg = a.nb;
        a.yend = a.nb + a.ny;
        a.zorg = a.nb;
        a.zend = a.nb + a.nz;
    } else {
        a.xorg = a.yorg = a.zorg = 0;
        a.xend = a.NX;
        a.yend = a.NY;
        a.zend = a.NZ;
    }
}

cudaError_t launch_stencil(int radius, int mode, const StepArgs& a, cudaStream_t s);
// the same step with TMA plane loads (tuning variants 2 and 3); status: device status word
// tile_rows: 16 (256-thread blocks) or 8 (128-thread blocks)
cudaError_t launch_stencil_tma(int radius, int mode, const StepArgs& a, int* status,
                               cudaStream_t s, int tile_rows = 16);
bool tma_available();
int auto_zchunk(int radius, int NX, int NY, int NZ);

// ---- small kernels (aux.cu) -------------------------------------------------
struct Geometry {
    int NX, NY, NZ, nb, nx, ny, nz;
};

// sponge factor g = gx gy gz of padded cell i
__device__ __forceinline__ float sponge_at(const Geometry& G, const float* gx, const float* gy,
                                           const float* gz, long long i) {
    const long long plane = (long long)G.NX * G.NY;
    const int z = (int)(i / plane);
    const int y = (int)((i % plane) / G.NX);
    const int x = (int)(i % G.NX);
    return gx[x] * gy[y] * gz[z];
}

cudaError_t launch_sponge(const Geometry& G, float* gx, float* gy, float* gz, cudaStream_t s);
cudaError_t launch_wavelet(int nt, double dt, double f0, double t0, float* w, cudaStream_t s);
cudaError_t launch_model_prep(const Geometry& G, const float* vel, int squared, double dt,
                              float* c, unsigned int* vmax_bits, int* bad, cudaStream_t s);
// forward step n: gather d[n-1] = u_cur[rec] (if data_row), then pre-adjust
// u_prev[s] -= c_s w / (dx^3 g_s^2) so that the stencil adds c_s w / dx^3.
cudaError_t launch_fwd_aux(const Geometry& G, const float* u_cur, float* u_prev,
                           const float* c, const float* gx, const float* gy,
                           const float* gz, const int32_t* rec, int nrec,
                           float* data_row, long long src, const float* w_n,
                           float inv_dx3, int* status, cudaStream_t s);
// backward step m: pre-adjust mu_prev[rec] -= c r / (dx^3 g) (if r_row) so
// that the stencil adds c g r / dx^3; record the source trace of mu_cur and
// the source term of the gradient (if requested).
cudaError_t launch_bwd_aux(const Geometry& G, const float* mu_cur, float* mu_prev,
                           const float* c, const float* gx, const float* gy,
                           const float* gz, const int32_t* rec, int nrec,
                           const float* r_row, long long src, float* src_adj_slot,
                           float* grad_acc, const float* w_n, float inv_dx3,
                           int* status, cudaStream_t s);
cudaError_t launch_image_finalize(const Geometry& G, const float* slab, float* image,
                                  cudaStream_t s);
cudaError_t launch_grad_finalize(const Geometry& G, const float* acc, const float* c,
                                 double dx3, double dt2, float* grad_v2, cudaStream_t s);
cudaError_t launch_misfit(const float* d, const float* obs, long long n, float* resid,
                          double* J, cudaStream_t s);
// decimated storage (the non-learned 8x scheme): keep every other model
// sample per axis of a padded field into coarse [(nz+1)/2][(ny+1)/2][(nx+1)/2];
// reconstruct the model region of a snapshot slab by linear interpolation
cudaError_t launch_decimate(const Geometry& G, const float* u, float* coarse, cudaStream_t s);
cudaError_t launch_upsample(const Geometry& G, const float* coarse, float* slab, cudaStream_t s);
// off-grid source and receivers (offgrid.cu): the same steps as
// launch_fwd_aux / launch_bwd_aux with each point spread over its tap table
// (taps[0] the source, taps[1 .. nrec] the receivers)
cudaError_t launch_fwd_aux_off(const Geometry& G, const float* u_cur, float* u_prev,
                               const float* c, const float* gx, const float* gy,
                               const float* gz, const rtm_point_taps* taps, int nrec,
                               float* data_row, const float* w_n, float inv_dx3, int* status,
                               cudaStream_t s);
cudaError_t launch_bwd_aux_off(const Geometry& G, const float* mu_cur, float* mu_prev,
                               const float* c, const float* gx, const float* gy,
                               const float* gz, const rtm_point_taps* taps, int nrec,
                               const float* r_row, float* src_adj_slot, float inv_dx3,
                               int* status, cudaStream_t s);
// post-run check: any non-finite value among n floats sets *status to
// RTM_ERR_NUMERIC (unless another error is already recorded)
cudaError_t launch_finite_scan(const float* f, long long n, int* status, cudaStream_t s);
// imaging-condition variants: source illumination (+= u^2 of a snapshot
// slab's model columns), illumination-normalised image, Laplacian filter
struct LapWeights {
    int r;
    float a[kMaxRadius + 1];  // a[0] = 3 a0 / dx^2, a[k] = a_k / dx^2
};
// boundary band of the model region (band.cuh): gather it from a padded
// field into band storage (to_field = 0) or scatter it back (to_field = 1)
cudaError_t launch_band_copy(const Geometry& G, int r, float* field, float* band, int to_field,
                             cudaStream_t s);
// illum += u^2 over the model region; u: the model slab, or a padded field (padded = 1)
cudaError_t launch_illum_add(const Geometry& G, const float* slab, float* illum, int padded,
                             cudaStream_t s);
cudaError_t launch_image_normalize(const float* image, const float* illum, long long n,
                                   unsigned int* max_bits, float eps_rel, float* out,
                                   cudaStream_t s);
cudaError_t launch_image_laplacian(const float* image, int nx, int ny, int nz,
                                   const LapWeights& w, float* out, cudaStream_t s);

// sets the thread-local message of rtm_last_error() and returns code
int set_error(int code, const char* fmt, ...);
// plane-load variant chosen by rtm_set_tuning for a radius (0: automatic)
int tuning_variant(int radius);
// z-slab height chosen by rtm_set_tuning for a radius (0: automatic); with a
// mode, that mode's height from rtm_set_tuning_mode where one is set
int tuning_zchunk(int radius, int mode = -1);
// the plane armed by rtm_set_test_stall for a kernel (RTM_STALL_*), or -1;
// taking it disarms it, so only the next launch stalls
int take_test_stall(int kernel);

}  // namespace rtm
