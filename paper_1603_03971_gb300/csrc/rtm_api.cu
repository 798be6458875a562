// C ABI of librtm: argument validation, workspace layout and the time loops
// of forward modelling, receiver propagation with imaging, the gradient and
// the end-to-end shot from host buffers.

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/rtm.h"
#include "ae_internal.h"
#include "band.cuh"
#include "revolve.h"
#include "rtm_internal.h"

using namespace rtm;

namespace {

thread_local std::string g_err;

rtm_status fail(rtm_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CU(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(RTM_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));   \
    } while (0)

#define CHECK(expr)                          \
    do {                                     \
        rtm_status s_ = (expr);              \
        if (s_ != RTM_OK) return s_;         \
    } while (0)

// largest stable vmax dt / dx: 2 / sqrt(3 |S(pi)|), S(pi) = a0 + 2 sum (-1)^k a_k
double stability_limit(int r) {
    double a[kMaxRadius + 1];
    stencil_weights(r, a);
    double s = a[0];
    for (int k = 1; k <= r; k++) s += 2.0 * ((k % 2) ? -a[k] : a[k]);
    return 2.0 / sqrt(3.0 * fabs(s));
}

// ---- tuning, timing and counters ---------------------------------------------
std::mutex g_mu;
int g_zchunk[kMaxRadius + 1] = {0};
// per stencil mode (statistics slot): slab height, 0 = the radius's general one
int g_zchunk_mode[kMaxRadius + 1][MODE_COUNT] = {{0}};
int g_variant[kMaxRadius + 1] = {0};
// one-shot stalls armed by rtm_set_test_stall (RTM_STALL_*), -1 = none
constexpr int kStallKernels = 2;
std::atomic<int> g_test_stall[kStallKernels] = {{-1}, {-1}};
bool g_timing = false;
rtm_stats g_stats;

struct PendingTiming {
    cudaEvent_t a, b;
    int mode;
    double bytes;
};

struct Timer {
    std::vector<PendingTiming> pending;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t get() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    rtm_status drain(cudaStream_t s) {
        if (pending.empty()) return RTM_OK;
        CU(cudaStreamSynchronize(s));
        std::lock_guard<std::mutex> lk(g_mu);
        for (auto& p : pending) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
                g_stats.stencil_ms[p.mode] += ms;
                g_stats.stencil_bytes[p.mode] += p.bytes;
            }
            pool.push_back(p.a);
            pool.push_back(p.b);
        }
        pending.clear();
        return RTM_OK;
    }
};
thread_local Timer t_timer;

void count_launch(int n = 1) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_stats.launches += n;
}

// ---- workspace layout ----------------------------------------------------------
constexpr size_t kAlign = 256;
constexpr size_t kStatusBytes = 256;  // status word at 0, model-prep reduction at 16,
                                      // image-filter maximum at 32
size_t up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Layout {
    size_t status = 0, wavelet = 0, gx = 0, gy = 0, gz = 0;
    size_t f[2] = {0, 0}, m[2] = {0, 0};
    size_t img = 0, grad = 0;
    size_t ckpt = 0, nckpt = 0;
    size_t snap = 0, nsnap = 0, snap_elems = 0;
    // learned storage: one latent and one scale per imaging step, codec scratch
    size_t latent = 0, latent_bytes = 0, scales = 0, ae_h = 0, ae_scalars = 0;
    // boundary storage: the model region's band of the states u^1 .. u^{nt-2}
    size_t band = 0, nband = 0, nbands = 0;
    size_t total = 0;
};

struct Dims {
    int NX, NY, NZ;
    size_t N, slab, nmodel;
};

Dims dims_of(const rtm_params* p) {
    Dims d;
    d.NX = p->nx + 2 * p->nb;
    d.NY = p->ny + 2 * p->nb;
    d.NZ = p->nz + 2 * p->nb;
    d.N = (size_t)d.NX * d.NY * d.NZ;
    d.slab = (size_t)p->nz * p->ny * d.NX;
    d.nmodel = (size_t)p->nx * p->ny * p->nz;
    return d;
}

Layout layout_of(const rtm_params* p) {
    const Dims d = dims_of(p);
    Layout L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += up(bytes);
        return o;
    };
    L.status = take(kStatusBytes);
    L.wavelet = take(sizeof(float) * (size_t)p->nt);
    L.gx = take(sizeof(float) * d.NX);
    L.gy = take(sizeof(float) * d.NY);
    L.gz = take(sizeof(float) * d.NZ);
    const size_t fb = sizeof(float) * d.N;
    L.f[0] = take(fb);
    L.f[1] = take(fb);
    L.m[0] = take(fb);
    L.m[1] = take(fb);
    if (p->want_grad) {
        L.grad = take(fb);
        L.snap_elems = d.N;
    } else {
        L.img = take(sizeof(float) * d.slab);
        L.snap_elems = d.slab;
    }
    if (p->storage == RTM_STORE_DECIMATED) {
        // one float32 coarse snapshot per imaging step, one decode slab plus
        // the exact window's slabs
        const size_t nlat = (size_t)(p->nt / p->image_every);
        L.latent_bytes = up(sizeof(float) * (size_t)((p->nx + 1) / 2) * ((p->ny + 1) / 2) *
                            ((p->nz + 1) / 2));
        L.latent = take(L.latent_bytes * (nlat ? nlat : 1));
        const size_t nwin = (size_t)(p->ckpt_every / p->image_every);
        L.nsnap = nwin > 1 ? nwin : 1;
    } else if (p->storage == RTM_STORE_LEARNED) {
        const size_t nlat = (size_t)(p->nt / p->image_every);
        L.latent_bytes = up((size_t)(p->nx / 4) * (p->ny / 4) * (p->nz / 4) * 16 * 2);
        L.latent = take(L.latent_bytes * (nlat ? nlat : 1));
        L.scales = take(sizeof(float) * (nlat ? nlat : 1));
        L.ae_h = take((size_t)(p->nx / 2) * (p->ny / 2) * (p->nz / 2) * 32 * 2);
        L.ae_scalars = take(256);
        // one decode slab; an exact window of ckpt_every steps needs one slab
        // per imaging step in it
        const size_t nwin = (size_t)(p->ckpt_every / p->image_every);
        L.nsnap = nwin > 1 ? nwin : 1;
    } else if (p->storage == RTM_STORE_ALL) {
        L.nsnap = p->want_grad ? (size_t)p->nt : (size_t)(p->nt / p->image_every);
    } else if (p->storage == RTM_STORE_REVOLVE) {
        const int M = p->nt / (p->image_every > 0 ? p->image_every : 1);
        L.nckpt = (size_t)(p->ckpt_every < M ? p->ckpt_every : M);
        L.ckpt = take(2 * fb * L.nckpt);
        L.nsnap = 1;  // the snapshot of the state being delivered
    } else if (p->storage == RTM_STORE_BOUNDARY) {
        // imaging reads the reconstructed field in place: no snapshot slab
        L.nband = (size_t)band_cells(p->nx, p->ny, p->nz, p->radius);
        L.nbands = p->nt > 2 ? (size_t)(p->nt - 2) : 0;
        L.band = take(sizeof(float) * L.nband * (L.nbands ? L.nbands : 1));
        L.nsnap = 0;
    } else {
        const int k = p->ckpt_every;
        const int nseg = (p->nt + k - 1) / k;
        L.nckpt = (size_t)(nseg > 1 ? nseg - 1 : 0);
        L.ckpt = take(2 * fb * L.nckpt);
        L.nsnap = (size_t)k;
    }
    if (p->storage != RTM_STORE_BOUNDARY)
        L.snap = take(sizeof(float) * L.snap_elems * (L.nsnap ? L.nsnap : 1));
    L.total = off;
    return L;
}

rtm_status validate(const rtm_params* p) {
    if (!p) return fail(RTM_ERR_INVALID, "params is NULL");
    if (p->nx < 1 || p->ny < 1 || p->nz < 1)
        return fail(RTM_ERR_INVALID, "model grid %dx%dx%d must be positive", p->nx, p->ny, p->nz);
    if (p->nb < 0) return fail(RTM_ERR_INVALID, "sponge width %d < 0", p->nb);
    if (p->radius != 4 && p->radius != 8)
        return fail(RTM_ERR_UNSUPPORTED, "stencil radius %d (4 or 8 supported)", p->radius);
    if (p->nt < 1) return fail(RTM_ERR_INVALID, "nt %d < 1", p->nt);
    if (!(p->dx > 0.0) || !(p->dt > 0.0) || !isfinite(p->dx) || !isfinite(p->dt))
        return fail(RTM_ERR_INVALID, "dx and dt must be positive and finite");
    if (!(p->f0 > 0.0) || !isfinite(p->f0) || !isfinite(p->t0))
        return fail(RTM_ERR_INVALID, "f0 must be positive, t0 finite");
    const long long NX = (long long)p->nx + 2LL * p->nb;
    const long long NY = (long long)p->ny + 2LL * p->nb;
    const long long NZ = (long long)p->nz + 2LL * p->nb;
    if (NX % 4 != 0)
        return fail(RTM_ERR_INVALID,
                    "padded x extent nx + 2 nb = %lld must be a multiple of 4 (16-byte rows)", NX);
    if (NX > (1LL << 24) || NY > 65535LL * 16 || NZ > (1LL << 24) || NX * NY > (1LL << 31))
        return fail(RTM_ERR_INVALID, "padded grid %lldx%lldx%lld too large", NX, NY, NZ);
    if (p->src_x < -p->nb || p->src_x >= p->nx + p->nb || p->src_y < -p->nb ||
        p->src_y >= p->ny + p->nb || p->src_z < -p->nb || p->src_z >= p->nz + p->nb)
        return fail(RTM_ERR_INVALID, "source (%d,%d,%d) outside the padded grid", p->src_x,
                    p->src_y, p->src_z);
    if (p->nrec < 0) return fail(RTM_ERR_INVALID, "nrec %d < 0", p->nrec);
    if (p->storage != RTM_STORE_ALL && p->storage != RTM_STORE_CKPT &&
        p->storage != RTM_STORE_LEARNED && p->storage != RTM_STORE_REVOLVE &&
        p->storage != RTM_STORE_BOUNDARY && p->storage != RTM_STORE_DECIMATED)
        return fail(RTM_ERR_INVALID, "storage %d unknown", p->storage);
    if (p->storage == RTM_STORE_BOUNDARY) {
        if (p->want_grad)
            return fail(RTM_ERR_INVALID, "boundary storage serves imaging, not the gradient");
        const int r2 = 2 * p->radius;
        if (p->nx <= r2 || p->ny <= r2 || p->nz <= r2)
            return fail(RTM_ERR_INVALID,
                        "boundary storage needs model sides above 2 r = %d (got %dx%dx%d)", r2,
                        p->nx, p->ny, p->nz);
    }
    if (p->storage == RTM_STORE_REVOLVE) {
        if (p->want_grad)
            return fail(RTM_ERR_INVALID, "binomial checkpointing serves imaging, not the gradient");
        if (p->ckpt_every < 0) return fail(RTM_ERR_INVALID, "checkpoint slots %d < 0", p->ckpt_every);
        if (p->image_every >= 1 && revolve_cost(p->nt / p->image_every, p->ckpt_every) < 0)
            return fail(RTM_ERR_UNSUPPORTED,
                        "binomial schedule for %d imaging steps and %d slots exceeds the planning limit",
                        p->nt / p->image_every, p->ckpt_every);
    }
    if (p->storage == RTM_STORE_LEARNED) {
        if (p->ckpt_every < 0 || p->ckpt_every > p->nt)
            return fail(RTM_ERR_INVALID, "exact window %d outside [0, nt]", p->ckpt_every);
        if (p->nx % 4 || p->ny % 4 || p->nz % 4)
            return fail(RTM_ERR_INVALID, "learned storage needs model sides that are multiples of 4");
        if (p->want_grad)
            return fail(RTM_ERR_INVALID, "learned storage serves imaging, not the gradient");
    }
    if (p->storage == RTM_STORE_DECIMATED) {
        if (p->ckpt_every < 0 || p->ckpt_every > p->nt)
            return fail(RTM_ERR_INVALID, "exact window %d outside [0, nt]", p->ckpt_every);
        if (p->want_grad)
            return fail(RTM_ERR_INVALID, "decimated storage serves imaging, not the gradient");
    }
    if (p->storage == RTM_STORE_CKPT && p->ckpt_every < 1)
        return fail(RTM_ERR_INVALID, "ckpt_every %d < 1", p->ckpt_every);
    if (p->image_every < 1) return fail(RTM_ERR_INVALID, "image_every %d < 1", p->image_every);
    if (p->want_grad != 0 && p->want_grad != 1)
        return fail(RTM_ERR_INVALID, "want_grad must be 0 or 1");
    if (p->want_grad && p->image_every != 1)
        return fail(RTM_ERR_INVALID, "the gradient needs image_every = 1");
    return RTM_OK;
}

rtm_status check_ws(const rtm_params* p, void* ws, size_t bytes) {
    if (!ws) return fail(RTM_ERR_WORKSPACE, "workspace is NULL");
    if ((uintptr_t)ws % kAlign) return fail(RTM_ERR_WORKSPACE, "workspace not 256-byte aligned");
    const size_t need = layout_of(p).total;
    if (bytes < need)
        return fail(RTM_ERR_WORKSPACE, "workspace %zu bytes, %zu needed", bytes, need);
    return RTM_OK;
}

bool aligned16(const void* q) { return ((uintptr_t)q % 16) == 0; }

// ---- per-call context ----------------------------------------------------------
struct Ctx {
    const rtm_params* p;
    Dims d;
    Layout L;
    Geometry G;
    char* ws;
    cudaStream_t s;
    StepArgs base;
    long long src;
    float inv_dx3;
    int variant;
    const float* ae = nullptr;  // codec parameters (learned storage)
    float* illum = nullptr;     // source illumination, model grid (+=), or NULL
    bool snap_padded = false;   // imaging snapshots are padded fields (boundary storage)
    int zchunk_mode[MODE_COUNT] = {0};  // per-mode slab heights (0: base.zchunk)
    const rtm_point_taps* taps = nullptr;  // off-grid source and receivers, or NULL

    float* at(size_t off) const { return reinterpret_cast<float*>(ws + off); }
    float* coarse_slot(size_t k) const {
        return reinterpret_cast<float*>(ws + L.latent + k * L.latent_bytes);
    }
    ae::bf16* latent_slot(size_t k) const {
        return reinterpret_cast<ae::bf16*>(ws + L.latent + k * L.latent_bytes);
    }
    // the model region of a padded field
    ae::Vol field_view(float* f) const {
        const long long NX = d.NX, NY = d.NY;
        return ae::Vol{f + ((long long)p->nb * NY + p->nb) * NX + p->nb, NX, NX * NY, p->nx, p->ny,
                       p->nz};
    }
    ae::Vol model_view(float* slab) const {
        return ae::Vol{slab + p->nb, (long long)d.NX, (long long)d.NX * p->ny, p->nx, p->ny, p->nz};
    }
    int* status() const { return reinterpret_cast<int*>(ws + L.status); }
    float* wav() const { return at(L.wavelet); }
    float* snap_slot(size_t k) const { return at(L.snap) + k * L.snap_elems; }
    float* ckpt_field(size_t j, int which) const {
        return at(L.ckpt) + ((j - 1) * 2 + which) * d.N;
    }
    // band of state u^m, 1 <= m <= nt - 2 (boundary storage)
    float* band_of(int m) const { return at(L.band) + (size_t)(m - 1) * L.nband; }
};

rtm_status make_ctx(Ctx& C, const rtm_params* p, const float* c, void* ws, rtm_stream s) {
    cudaGetLastError();  // a stale error of earlier work must not be taken for ours
    C.p = p;
    C.d = dims_of(p);
    C.L = layout_of(p);
    C.G = Geometry{C.d.NX, C.d.NY, C.d.NZ, p->nb, p->nx, p->ny, p->nz};
    C.ws = reinterpret_cast<char*>(ws);
    C.s = reinterpret_cast<cudaStream_t>(s);
    C.src = ((long long)(p->src_z + p->nb) * C.d.NY + (p->src_y + p->nb)) * C.d.NX +
            (p->src_x + p->nb);
    C.inv_dx3 = (float)(1.0 / (p->dx * p->dx * p->dx));
    memset(&C.base, 0, sizeof C.base);
    step_weights(p->radius, p->dx, C.base.a);
    C.base.c = c;
    C.base.gx = C.at(C.L.gx);
    C.base.gy = C.at(C.L.gy);
    C.base.gz = C.at(C.L.gz);
    C.base.NX = C.d.NX;
    C.base.NY = C.d.NY;
    C.base.NZ = C.d.NZ;
    C.base.nb = p->nb;
    C.base.nx = p->nx;
    C.base.ny = p->ny;
    C.base.nz = p->nz;
    int zc, var;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        zc = g_zchunk[p->radius];
        var = g_variant[p->radius];
        for (int m = 0; m < MODE_COUNT; m++) C.zchunk_mode[m] = g_zchunk_mode[p->radius][m];
    }
    C.base.zchunk = zc > 0 ? zc : auto_zchunk(p->radius, C.d.NX, C.d.NY, C.d.NZ);
    if ((C.d.NZ + C.base.zchunk - 1) / C.base.zchunk > 65535)
        C.base.zchunk = (C.d.NZ + 65534) / 65535;  // grid.z limit
    // automatic: TMA plane loads wherever the driver provides tensor maps
    C.variant = var != 0 ? var : (tma_available() ? 2 : 1);
    C.snap_padded = p->storage == RTM_STORE_BOUNDARY;
    set_region(C.base, MODE_FWD);
    return RTM_OK;
}

double stencil_bytes(const Ctx& C, int mode) {
    const double N = (double)C.d.N, M = (double)C.d.nmodel;
    switch (mode) {
        case MODE_FWD: return 16.0 * N;
        case MODE_FWD_SNAP: return 16.0 * N + 4.0 * M;
        case MODE_BWD_IMAGE: return 16.0 * N + 12.0 * M;
        case MODE_FWD_LU: return 20.0 * N;
        case MODE_BWD_GRAD: return 28.0 * N;
        case MODE_REV: return 16.0 * M;
        default: return 0.0;
    }
}

rtm_status stencil(Ctx& C, int mode, const float* cur, float* prev, float* snap, float* acc,
                   double* sumsq = nullptr) {
    StepArgs a = C.base;
    a.u_cur = cur;
    a.u_prev = prev;
    a.snap = snap;
    a.acc = acc;
    a.sumsq = sumsq;
    // the statistics count the sum-of-squares forward step as a forward step
    const int slot = mode == MODE_FWD_SUMSQ ? MODE_FWD : mode;
    set_region(a, mode);
    // the reverse step covers the model region: its slabs are sized for its
    // own tiles (a slab height tuned for the padded grid can leave it a
    // nearly empty last wave)
    if (mode == MODE_REV)
        a.zchunk = auto_zchunk(C.p->radius, a.xend - a.xorg, a.yend - a.yorg, a.zend - a.zorg);
    // a slab height tuned for this mode (its statistics slot) wins
    if (C.zchunk_mode[slot] > 0) a.zchunk = C.zchunk_mode[slot];
    if ((a.zend - a.zorg + a.zchunk - 1) / a.zchunk > 65535)
        a.zchunk = (a.zend - a.zorg + 65534) / 65535;  // grid.z limit
    a.snap_padded = (mode == MODE_BWD_IMAGE && C.snap_padded) ? 1 : 0;
    bool timing;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        timing = g_timing;
        g_stats.launches += 1;
        g_stats.stencil_launches[slot] += 1;
    }
    if (timing) {
        PendingTiming t{t_timer.get(), t_timer.get(), slot, stencil_bytes(C, slot)};
        CU(cudaEventRecord(t.a, C.s));
        CU(C.variant >= 2 ? launch_stencil_tma(C.p->radius, mode, a, C.status(), C.s,
                                               C.variant == 3 ? 8 : 16)
                          : launch_stencil(C.p->radius, mode, a, C.s));
        CU(cudaEventRecord(t.b, C.s));
        t_timer.pending.push_back(t);
        if (t_timer.pending.size() >= 2048) CHECK(t_timer.drain(C.s));
    } else {
        CU(C.variant >= 2 ? launch_stencil_tma(C.p->radius, mode, a, C.status(), C.s,
                                               C.variant == 3 ? 8 : 16)
                          : launch_stencil(C.p->radius, mode, a, C.s));
    }
    return RTM_OK;
}

rtm_status prepare_tables(Ctx& C) {
    CU(launch_wavelet(C.p->nt, C.p->dt, C.p->f0, C.p->t0, C.wav(), C.s));
    CU(launch_sponge(C.G, C.at(C.L.gx), C.at(C.L.gy), C.at(C.L.gz), C.s));
    count_launch(2);
    return RTM_OK;
}

rtm_status fwd_aux(Ctx& C, const float* cur, float* prev, const int32_t* rec, float* data_row,
                   const float* w_n) {
    if (C.taps)
        CU(launch_fwd_aux_off(C.G, cur, prev, C.base.c, C.base.gx, C.base.gy, C.base.gz, C.taps,
                              C.p->nrec, data_row, w_n, C.inv_dx3, C.status(), C.s));
    else
        CU(launch_fwd_aux(C.G, cur, prev, C.base.c, C.base.gx, C.base.gy, C.base.gz, rec,
                          C.p->nrec, data_row, C.src, w_n, C.inv_dx3, C.status(), C.s));
    count_launch();
    return RTM_OK;
}

rtm_status bwd_aux(Ctx& C, const float* mcur, float* mprev, const int32_t* rec,
                   const float* r_row, float* src_adj_slot, float* grad_acc, const float* w_n) {
    if (C.taps)  // imaging only: no gradient source term
        CU(launch_bwd_aux_off(C.G, mcur, mprev, C.base.c, C.base.gx, C.base.gy, C.base.gz,
                              C.taps, C.p->nrec, r_row, src_adj_slot, C.inv_dx3, C.status(),
                              C.s));
    else
        CU(launch_bwd_aux(C.G, mcur, mprev, C.base.c, C.base.gx, C.base.gy, C.base.gz, rec,
                          C.p->nrec, r_row, C.src, src_adj_slot, grad_acc, w_n, C.inv_dx3,
                          C.status(), C.s));
    count_launch();
    return RTM_OK;
}

// forward modelling; leaves snapshots (store-all) or checkpoints in the workspace
rtm_status run_forward(Ctx& C, const int32_t* rec, float* data, float* u_last) {
    const rtm_params* p = C.p;
    const size_t fb = sizeof(float) * C.d.N;
    // a forward pass starts a pipeline: clear the device status word
    CU(cudaMemsetAsync(C.status(), 0, sizeof(int), C.s));
    float* prev = C.at(C.L.f[0]);
    float* cur = C.at(C.L.f[1]);
    CU(cudaMemsetAsync(prev, 0, fb, C.s));
    CU(cudaMemsetAsync(cur, 0, fb, C.s));
    CHECK(prepare_tables(C));
    const int k = p->ckpt_every, ie = p->image_every;
    for (int n = 0; n < p->nt; n++) {
        if (p->storage == RTM_STORE_CKPT && n > 0 && n % k == 0) {
            const size_t j = (size_t)(n / k);
            CU(cudaMemcpyAsync(C.ckpt_field(j, 0), prev, fb, cudaMemcpyDeviceToDevice, C.s));
            CU(cudaMemcpyAsync(C.ckpt_field(j, 1), cur, fb, cudaMemcpyDeviceToDevice, C.s));
        }
        float* row = (data && n >= 1) ? data + (size_t)(n - 1) * p->nrec : nullptr;
        CHECK(fwd_aux(C, cur, prev, rec, row, C.wav() + n));
        int mode = MODE_FWD;
        float* snap = nullptr;
        if (p->storage == RTM_STORE_ALL) {
            if (p->want_grad) {
                mode = MODE_FWD_LU;
                snap = C.snap_slot((size_t)n);
            } else if ((n + 1) % ie == 0) {
                mode = MODE_FWD_SNAP;
                snap = C.snap_slot((size_t)((n + 1) / ie - 1));
            }
        }
        // learned storage: the step that writes a coded snapshot also sums
        // its squares for the encoder's scale (no separate pass over it)
        const bool code = p->storage == RTM_STORE_LEARNED && (n + 1) % ie == 0 &&
                          n + 1 > p->ckpt_every;
        const bool decim = p->storage == RTM_STORE_DECIMATED && (n + 1) % ie == 0 &&
                           n + 1 > p->ckpt_every;
        auto* scal = reinterpret_cast<ae::AeScalars*>(C.at(C.L.ae_scalars));
        if (code) {
            CU(cudaMemsetAsync(&scal->sumsq, 0, sizeof(double), C.s));
            mode = MODE_FWD_SUMSQ;
        }
        CHECK(stencil(C, mode, cur, prev, snap, nullptr, code ? &scal->sumsq : nullptr));
        if (p->storage == RTM_STORE_BOUNDARY && n + 1 <= p->nt - 2) {
            // the band of u^{n+1} (now in prev)
            CU(launch_band_copy(C.G, p->radius, prev, C.band_of(n + 1), 0, C.s));
            count_launch();
        }
        if (decim) {  // u^{n+1} (now in prev): every other sample per axis
            CU(launch_decimate(C.G, prev, C.coarse_slot((size_t)((n + 1) / ie - 1)), C.s));
            count_launch();
        }
        if (code) {
            // the encoder reads u^{n+1} (now in prev) in place: no snapshot copy
            const size_t k = (size_t)((n + 1) / ie - 1);
            CU(ae_encode(C.ae, C.field_view(prev), reinterpret_cast<ae::bf16*>(C.at(C.L.ae_h)),
                         C.latent_slot(k), scal, C.at(C.L.scales) + k, C.status(), C.s,
                         false, true));
            count_launch(2);  // scale, encoder
        }
        float* t = prev;
        prev = cur;
        cur = t;
    }
    if (data)
        CHECK(fwd_aux(C, cur, prev, rec, data + (size_t)(p->nt - 1) * p->nrec, nullptr));
    if (u_last) {
        CU(cudaMemcpyAsync(u_last, prev, fb, cudaMemcpyDeviceToDevice, C.s));
        CU(cudaMemcpyAsync(u_last + C.d.N, cur, fb, cudaMemcpyDeviceToDevice, C.s));
    }
    // a non-finite value, once it appears, stays in the newest state: one
    // scan of u^{nt} flags a run that blew up (rtm_check reports it)
    CU(launch_finite_scan(cur, (long long)C.d.N, C.status(), C.s));
    count_launch();
    return RTM_OK;
}

// binomial checkpointing: the source states the imaging steps need, in
// reverse order, from a schedule of forward recomputation, slot stores and
// restores (revolve.h); backward steps run as their states are delivered
template <class BackStep>
rtm_status run_revolve(Ctx& C, const int32_t* rec, BackStep& back_step) {
    const rtm_params* p = C.p;
    const int ie = p->image_every;
    const int M = p->nt / ie;
    std::vector<RevolveAction> plan;
    if (!revolve_schedule(M, p->ckpt_every, plan))
        return fail(RTM_ERR_UNSUPPORTED, "binomial schedule over the planning limit");
    const size_t fb = sizeof(float) * C.d.N;
    float* fp = C.at(C.L.f[0]);  // u^{n-1} of the working pair
    float* fc = C.at(C.L.f[1]);  // u^n
    float* slab = C.snap_slot(0);
    const size_t row = sizeof(float) * (size_t)p->ny * C.d.NX;  // model rows of one plane
    int m_next = p->nt;  // next backward step
    for (const RevolveAction& A : plan) {
        switch (A.op) {
            case REV_RESTORE:
                if (A.a < 0) {
                    CU(cudaMemsetAsync(fp, 0, fb, C.s));
                    CU(cudaMemsetAsync(fc, 0, fb, C.s));
                } else {
                    CU(cudaMemcpyAsync(fp, C.ckpt_field((size_t)A.a + 1, 0), fb,
                                       cudaMemcpyDeviceToDevice, C.s));
                    CU(cudaMemcpyAsync(fc, C.ckpt_field((size_t)A.a + 1, 1), fb,
                                       cudaMemcpyDeviceToDevice, C.s));
                }
                break;
            case REV_ADVANCE:
                for (int n = A.a * ie; n < A.b * ie; n++) {
                    CHECK(fwd_aux(C, fc, fp, rec, nullptr, C.wav() + n));
                    const bool snap = A.c && n == A.b * ie - 1;
                    CHECK(stencil(C, snap ? MODE_FWD_SNAP : MODE_FWD, fc, fp, snap ? slab : nullptr,
                                  nullptr));
                    float* t = fp;
                    fp = fc;
                    fc = t;
                }
                break;
            case REV_STORE:
                CU(cudaMemcpyAsync(C.ckpt_field((size_t)A.a + 1, 0), fp, fb,
                                   cudaMemcpyDeviceToDevice, C.s));
                CU(cudaMemcpyAsync(C.ckpt_field((size_t)A.a + 1, 1), fc, fb,
                                   cudaMemcpyDeviceToDevice, C.s));
                break;
            case REV_DELIVER: {
                const int m_img = A.a * ie;
                if (A.b >= 0) {  // u^m of a stored pair: its model rows into the slab
                    const float* u = C.ckpt_field((size_t)A.b + 1, 1) +
                                     ((size_t)p->nb * C.d.NY + p->nb) * C.d.NX;
                    CU(cudaMemcpy2DAsync(slab, row, u, sizeof(float) * (size_t)C.d.NY * C.d.NX,
                                         row, (size_t)p->nz, cudaMemcpyDeviceToDevice, C.s));
                }
                for (; m_next > m_img; m_next--) {
                    if (m_next % ie == 0) return fail(RTM_ERR_STATE, "schedule skipped step %d", m_next);
                    CHECK(back_step(m_next, nullptr));
                }
                CHECK(back_step(m_img, slab));
                m_next = m_img - 1;
                break;
            }
            default:
                break;
        }
    }
    for (; m_next >= 1; m_next--) {
        if (m_next % ie == 0) return fail(RTM_ERR_STATE, "schedule skipped step %d", m_next);
        CHECK(back_step(m_next, nullptr));
    }
    return RTM_OK;
}

// receiver propagation, imaging (grad = false) or gradient accumulation (grad = true)
rtm_status run_backward(Ctx& C, const int32_t* rec, const float* rdata, float* src_adj,
                        bool grad) {
    const rtm_params* p = C.p;
    const size_t fb = sizeof(float) * C.d.N;
    float* mprev = C.at(C.L.m[0]);
    float* mcur = C.at(C.L.m[1]);
    float* acc = grad ? C.at(C.L.grad) : C.at(C.L.img);
    CU(cudaMemsetAsync(mprev, 0, fb, C.s));
    CU(cudaMemsetAsync(mcur, 0, fb, C.s));
    CU(cudaMemsetAsync(acc, 0, sizeof(float) * (grad ? C.d.N : C.d.slab), C.s));
    CHECK(prepare_tables(C));
    const int ie = p->image_every;

    auto back_step = [&](int m, float* snap) -> rtm_status {
        float* adj = (src_adj && m < p->nt) ? src_adj + m : nullptr;
        float* gacc = (grad && m < p->nt) ? acc : nullptr;
        CHECK(bwd_aux(C, mcur, mprev, rec, rdata + (size_t)(m - 1) * p->nrec, adj, gacc,
                      C.wav() + (m < p->nt ? m : 0)));
        int mode = MODE_FWD;
        if (grad) mode = MODE_BWD_GRAD;
        else if (m % ie == 0) mode = MODE_BWD_IMAGE;
        CHECK(stencil(C, mode, mcur, mprev, mode == MODE_FWD ? nullptr : snap,
                      mode == MODE_FWD ? nullptr : acc));
        if (mode == MODE_BWD_IMAGE && C.illum) {
            CU(launch_illum_add(C.G, snap, C.illum, C.snap_padded ? 1 : 0, C.s));
            count_launch();
        }
        float* t = mprev;
        mprev = mcur;
        mcur = t;
        return RTM_OK;
    };

    if (p->storage == RTM_STORE_LEARNED || p->storage == RTM_STORE_DECIMATED) {
        const int W = p->ckpt_every;  // exact window: steps 1..W recomputed, not coded
        float* slab = C.snap_slot(0);
        // columns outside the model stay finite (the decoders write model columns)
        CU(cudaMemsetAsync(slab, 0, sizeof(float) * C.d.slab, C.s));
        for (int m = p->nt; m > W; m--) {
            if (m % ie == 0) {
                const size_t k = (size_t)(m / ie - 1);
                if (p->storage == RTM_STORE_DECIMATED)
                    CU(launch_upsample(C.G, C.coarse_slot(k), slab, C.s));
                else
                    CU(ae_decode(C.ae, C.latent_slot(k), C.at(C.L.scales) + k,
                                 C.model_view(slab), nullptr, C.status(), C.s));
                count_launch(1);
            }
            CHECK(back_step(m, slab));
        }
        if (W > 0) {  // checkpoint-recompute fallback from the zero initial state
            float* rp = C.at(C.L.f[0]);
            float* rc = C.at(C.L.f[1]);
            CU(cudaMemsetAsync(rp, 0, fb, C.s));
            CU(cudaMemsetAsync(rc, 0, fb, C.s));
            for (int n = 0; n < W; n++) {
                CHECK(fwd_aux(C, rc, rp, rec, nullptr, C.wav() + n));
                const bool snap = (n + 1) % ie == 0;
                CHECK(stencil(C, snap ? MODE_FWD_SNAP : MODE_FWD, rc, rp,
                              snap ? C.snap_slot((size_t)((n + 1) / ie - 1)) : nullptr, nullptr));
                float* t = rp;
                rp = rc;
                rc = t;
            }
            for (int m = W; m >= 1; m--)
                CHECK(back_step(m, m % ie == 0 ? C.snap_slot((size_t)(m / ie - 1)) : nullptr));
        }
    } else if (p->storage == RTM_STORE_REVOLVE) {
        CHECK(run_revolve(C, rec, back_step));
    } else if (p->storage == RTM_STORE_BOUNDARY) {
        // the forward run leaves u^{nt} in f[(nt + 1) % 2] and u^{nt-1} in
        // f[nt % 2]; each earlier state is recovered in the model region by
        // the reverse step, in place over the state two steps later
        float* hi = C.at(C.L.f[(p->nt + 1) % 2]);  // u^{m+1}
        float* lo = C.at(C.L.f[p->nt % 2]);        // u^m
        CHECK(back_step(p->nt, p->nt % ie == 0 ? hi : nullptr));
        for (int m = p->nt - 1; m >= 1; m--) {
            if (m <= p->nt - 2) {
                // lo = u^{m+1}, hi = u^{m+2}: undo forward step m + 1 (its
                // source injection is undone by the same pre-adjustment)
                CHECK(fwd_aux(C, lo, hi, rec, nullptr, C.wav() + m + 1));
                CHECK(stencil(C, MODE_REV, lo, hi, nullptr, nullptr));
                // band cells: their stencils reach into the sponge; stored
                CU(launch_band_copy(C.G, p->radius, hi, C.band_of(m), 1, C.s));
                count_launch();
                float* t = lo;
                lo = hi;
                hi = t;
            }
            CHECK(back_step(m, m % ie == 0 ? lo : nullptr));
        }
    } else if (p->storage == RTM_STORE_ALL) {
        for (int m = p->nt; m >= 1; m--) {
            float* snap = nullptr;
            if (grad) snap = C.snap_slot((size_t)(m - 1));
            else if (m % ie == 0) snap = C.snap_slot((size_t)(m / ie - 1));
            CHECK(back_step(m, snap));
        }
    } else {
        const int k = p->ckpt_every;
        const int nseg = (p->nt + k - 1) / k;
        for (int j = nseg - 1; j >= 0; j--) {
            const int n0 = j * k, n1 = (n0 + k < p->nt) ? n0 + k : p->nt;
            float *rprev, *rcur;
            if (j == 0) {
                rprev = C.at(C.L.f[0]);
                rcur = C.at(C.L.f[1]);
                CU(cudaMemsetAsync(rprev, 0, fb, C.s));
                CU(cudaMemsetAsync(rcur, 0, fb, C.s));
            } else {
                rprev = C.ckpt_field((size_t)j, 0);
                rcur = C.ckpt_field((size_t)j, 1);
            }
            // recompute the segment from its checkpoint (in place)
            for (int n = n0; n < n1; n++) {
                CHECK(fwd_aux(C, rcur, rprev, rec, nullptr, C.wav() + n));
                int mode = MODE_FWD;
                float* snap = nullptr;
                if (grad) {
                    mode = MODE_FWD_LU;
                    snap = C.snap_slot((size_t)(n - n0));
                } else if ((n + 1) % ie == 0) {
                    mode = MODE_FWD_SNAP;
                    snap = C.snap_slot((size_t)(n - n0));
                }
                CHECK(stencil(C, mode, rcur, rprev, snap, nullptr));
                float* t = rprev;
                rprev = rcur;
                rcur = t;
            }
            for (int m = n1; m > n0; m--) CHECK(back_step(m, C.snap_slot((size_t)(m - 1 - n0))));
        }
    }
    // n = 0 terms: source trace and gradient source term of mu^1
    CHECK(bwd_aux(C, mcur, mprev, rec, nullptr, src_adj, grad ? acc : nullptr, C.wav()));
    // post-run scan of the accumulated image or gradient
    CU(launch_finite_scan(acc, (long long)(grad ? C.d.N : C.d.slab), C.status(), C.s));
    count_launch();
    return RTM_OK;
}

rtm_status finish(Ctx& C) {
    bool timing;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        timing = g_timing;
    }
    if (timing) CHECK(t_timer.drain(C.s));
    return RTM_OK;
}

rtm_status common_checks(const rtm_params* p, const float* d_c, const int32_t* d_rec, void* ws,
                         size_t ws_bytes) {
    CHECK(validate(p));
    CHECK(check_ws(p, ws, ws_bytes));
    if (!d_c) return fail(RTM_ERR_INVALID, "coefficient grid is NULL");
    if (!aligned16(d_c)) return fail(RTM_ERR_INVALID, "coefficient grid not 16-byte aligned");
    if (p->nrec > 0 && !d_rec) return fail(RTM_ERR_INVALID, "receiver array is NULL");
    return RTM_OK;
}

}  // namespace

// ---- stencil weights (closed form) -------------------------------------------
void rtm::stencil_weights(int r, double* a) {
    double fr = 1.0;
    for (int i = 2; i <= r; i++) fr *= i;
    double sum = 0.0;
    for (int k = 1; k <= r; k++) {
        double f_rmk = 1.0, f_rpk = 1.0;
        for (int i = 2; i <= r - k; i++) f_rmk *= i;
        for (int i = 2; i <= r + k; i++) f_rpk *= i;
        const double sign = (k % 2 == 1) ? 1.0 : -1.0;
        a[k] = 2.0 * sign * fr * fr / ((double)k * k * f_rmk * f_rpk);
        sum += a[k];
    }
    a[0] = -2.0 * sum;
}

void rtm::step_weights(int r, double dx, float* out) {
    double a[kMaxRadius + 1];
    stencil_weights(r, a);
    const double inv_dx2 = 1.0 / (dx * dx);
    out[0] = (float)(3.0 * a[0] * inv_dx2);
    for (int k = 1; k <= r; k++) out[k] = (float)(a[k] * inv_dx2);
}

int rtm::tuning_zchunk(int radius, int mode) {
    if (radius < 0 || radius > kMaxRadius) return 0;
    std::lock_guard<std::mutex> lk(g_mu);
    if (mode >= 0 && mode < MODE_COUNT && g_zchunk_mode[radius][mode] > 0)
        return g_zchunk_mode[radius][mode];
    return g_zchunk[radius];
}

int rtm::tuning_variant(int radius) {
    if (radius < 0 || radius > kMaxRadius) return 0;
    std::lock_guard<std::mutex> lk(g_mu);
    return g_variant[radius];
}

int rtm::take_test_stall(int kernel) {
    if (kernel < 0 || kernel >= kStallKernels) return -1;
    if (g_test_stall[kernel].load(std::memory_order_relaxed) < 0) return -1;
    return g_test_stall[kernel].exchange(-1);
}

int rtm::set_error(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

// ==== C ABI ======================================================================
extern "C" {

const char* rtm_version(void) { return "librtm 1.0 (sm_103a)"; }

const char* rtm_last_error(void) { return g_err.c_str(); }

rtm_status rtm_validate(const rtm_params* p) { return validate(p); }

size_t rtm_workspace_size(const rtm_params* p) {
    if (validate(p) != RTM_OK) return 0;
    return layout_of(p).total;
}

rtm_status rtm_model_prep(const rtm_params* p, const float* d_vel, int32_t vel_kind, float* d_c,
                          void* d_ws, size_t ws_bytes, rtm_stream stream) {
    CHECK(validate(p));
    if (!d_vel || !d_c) return fail(RTM_ERR_INVALID, "velocity or coefficient grid is NULL");
    if (!aligned16(d_vel) || !aligned16(d_c))
        return fail(RTM_ERR_INVALID, "velocity or coefficient grid not 16-byte aligned");
    if (vel_kind != RTM_VEL_V && vel_kind != RTM_VEL_V2)
        return fail(RTM_ERR_INVALID, "vel_kind %d unknown", vel_kind);
    if (!d_ws || ws_bytes < kStatusBytes) return fail(RTM_ERR_WORKSPACE, "workspace missing");
    if ((uintptr_t)d_ws % kAlign) return fail(RTM_ERR_WORKSPACE, "workspace not 256-byte aligned");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaGetLastError();
    const Dims d = dims_of(p);
    Geometry G{d.NX, d.NY, d.NZ, p->nb, p->nx, p->ny, p->nz};
    // reduction words in the status block of the workspace
    unsigned int* vmax = reinterpret_cast<unsigned int*>(reinterpret_cast<char*>(d_ws) + 16);
    int* bad = reinterpret_cast<int*>(reinterpret_cast<char*>(d_ws) + 20);
    CU(cudaMemsetAsync(vmax, 0, sizeof(unsigned int), s));
    CU(cudaMemsetAsync(bad, 0, sizeof(int), s));
    CU(launch_model_prep(G, d_vel, vel_kind == RTM_VEL_V2, p->dt, d_c, vmax, bad, s));
    count_launch();
    unsigned int h_vmax = 0;
    int h_bad = 0;
    CU(cudaMemcpyAsync(&h_vmax, vmax, sizeof h_vmax, cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(&h_bad, bad, sizeof h_bad, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (h_bad) return fail(RTM_ERR_NUMERIC, "velocity model has non-finite or non-positive values");
    float v2max;
    memcpy(&v2max, &h_vmax, sizeof v2max);
    const double vmax_v = sqrt((double)v2max);
    const double courant = vmax_v * p->dt / p->dx;
    const double lim = stability_limit(p->radius);
    if (courant > lim)
        return fail(RTM_ERR_CFL, "vmax dt / dx = %.6f exceeds the stability limit %.6f (r = %d)",
                    courant, lim, p->radius);
    return RTM_OK;
}

rtm_status rtm_forward(const rtm_params* p, const float* d_c, const int32_t* d_rec, float* d_data,
                       void* d_ws, size_t ws_bytes, float* d_u_last, rtm_stream stream) {
    CHECK(common_checks(p, d_c, d_rec, d_ws, ws_bytes));
    if (p->storage == RTM_STORE_LEARNED)
        return fail(RTM_ERR_STATE, "learned storage: use rtm_forward_learned");
    Ctx C;
    CHECK(make_ctx(C, p, d_c, d_ws, stream));
    CHECK(run_forward(C, d_rec, d_data, d_u_last));
    return finish(C);
}

rtm_status rtm_backward_image(const rtm_params* p, const float* d_c, const int32_t* d_rec,
                              const float* d_rdata, void* d_ws, size_t ws_bytes, float* d_image,
                              float* d_src_adj, rtm_stream stream) {
    CHECK(common_checks(p, d_c, d_rec, d_ws, ws_bytes));
    if (p->want_grad)
        return fail(RTM_ERR_STATE, "workspace prepared for the gradient (want_grad = 1)");
    if (p->storage == RTM_STORE_LEARNED)
        return fail(RTM_ERR_STATE, "learned storage: use rtm_backward_image_learned");
    if (!d_rdata && p->nrec > 0) return fail(RTM_ERR_INVALID, "receiver data is NULL");
    if (!d_image) return fail(RTM_ERR_INVALID, "image is NULL");
    Ctx C;
    CHECK(make_ctx(C, p, d_c, d_ws, stream));
    CHECK(run_backward(C, d_rec, d_rdata, d_src_adj, false));
    CU(launch_image_finalize(C.G, C.at(C.L.img), d_image, C.s));
    count_launch();
    return finish(C);
}

rtm_status rtm_shot(const rtm_params* p, const float* d_c, const int32_t* d_rec,
                    const float* d_dobs, float* d_data, void* d_ws, size_t ws_bytes,
                    float* d_image, rtm_stream stream) {
    CHECK(common_checks(p, d_c, d_rec, d_ws, ws_bytes));
    if (p->want_grad)
        return fail(RTM_ERR_STATE, "workspace prepared for the gradient (want_grad = 1)");
    if (p->storage == RTM_STORE_LEARNED)
        return fail(RTM_ERR_STATE, "learned storage: use rtm_shot_learned");
    if (!d_dobs && p->nrec > 0) return fail(RTM_ERR_INVALID, "observed data is NULL");
    if (!d_image) return fail(RTM_ERR_INVALID, "image is NULL");
    Ctx C;
    CHECK(make_ctx(C, p, d_c, d_ws, stream));
    CHECK(run_forward(C, d_rec, d_data, nullptr));
    CHECK(run_backward(C, d_rec, d_dobs, nullptr, false));
    CU(launch_image_finalize(C.G, C.at(C.L.img), d_image, C.s));
    count_launch();
    return finish(C);
}

static rtm_status offgrid_checks(const rtm_params* p, const float* d_c,
                                 const rtm_point_taps* d_taps, void* d_ws, size_t ws_bytes) {
    // the receivers come from the tap table: common_checks with a stand-in
    // receiver pointer
    CHECK(common_checks(p, d_c, reinterpret_cast<const int32_t*>(d_taps), d_ws, ws_bytes));
    if (!d_taps) return fail(RTM_ERR_INVALID, "tap table is NULL");
    if ((uintptr_t)d_taps % 16) return fail(RTM_ERR_INVALID, "tap table not 16-byte aligned");
    if (p->want_grad)
        return fail(RTM_ERR_STATE, "off-grid points serve modelling and imaging, not the gradient");
    if (p->storage == RTM_STORE_LEARNED)
        return fail(RTM_ERR_STATE, "off-grid points are not available with learned storage");
    return RTM_OK;
}

rtm_status rtm_forward_offgrid(const rtm_params* p, const float* d_c,
                               const rtm_point_taps* d_taps, float* d_data, void* d_ws,
                               size_t ws_bytes, float* d_u_last, rtm_stream stream) {
    CHECK(offgrid_checks(p, d_c, d_taps, d_ws, ws_bytes));
    Ctx C;
    CHECK(make_ctx(C, p, d_c, d_ws, stream));
    C.taps = d_taps;
    CHECK(run_forward(C, nullptr, d_data, d_u_last));
    return finish(C);
}

rtm_status rtm_shot_offgrid(const rtm_params* p, const float* d_c, const rtm_point_taps* d_taps,
                            const float* d_dobs, float* d_data, void* d_ws, size_t ws_bytes,
                            float* d_image, rtm_stream stream) {
    CHECK(offgrid_checks(p, d_c, d_taps, d_ws, ws_bytes));
    if (!d_dobs && p->nrec > 0) return fail(RTM_ERR_INVALID, "observed data is NULL");
    if (!d_image) return fail(RTM_ERR_INVALID, "image is NULL");
    Ctx C;
    CHECK(make_ctx(C, p, d_c, d_ws, stream));
    C.taps = d_taps;
    CHECK(run_forward(C, nullptr, d_data, nullptr));
    CHECK(run_backward(C, nullptr, d_dobs, nullptr, false));
    CU(launch_image_finalize(C.G, C.at(C.L.img), d_image, C.s));
    count_launch();
    return finish(C);
}

rtm_status rtm_grad(const rtm_params* p, const float* d_c, const int32_t* d_rec,
                    const float* d_resid, void* d_ws, size_t ws_bytes, float* d_grad_v2,
                    rtm_stream stream) {
    CHECK(common_checks(p, d_c, d_rec, d_ws, ws_bytes));
    if (!p->want_grad)
        return fail(RTM_ERR_STATE, "workspace prepared for imaging (want_grad = 0)");
    if (!d_resid && p->nrec > 0) return fail(RTM_ERR_INVALID, "residual is NULL");
    if (!d_grad_v2) return fail(RTM_ERR_INVALID, "gradient output is NULL");
    Ctx C;
    CHECK(make_ctx(C, p, d_c, d_ws, stream));
    CHECK(run_backward(C, d_rec, d_resid, nullptr, true));
    CU(launch_grad_finalize(C.G, C.at(C.L.grad), d_c, p->dx * p->dx * p->dx, p->dt * p->dt,
                            d_grad_v2, C.s));
    count_launch();
    return finish(C);
}

static rtm_status learned_checks(const rtm_params* p, const float* d_c, const int32_t* d_rec,
                                 const float* d_ae, void* d_ws, size_t ws_bytes) {
    CHECK(common_checks(p, d_c, d_rec, d_ws, ws_bytes));
    if (p->storage != RTM_STORE_LEARNED)
        return fail(RTM_ERR_STATE, "the learned calls need storage = RTM_STORE_LEARNED");
    if (!d_ae) return fail(RTM_ERR_INVALID, "codec parameters are NULL");
    return RTM_OK;
}

rtm_status rtm_forward_learned(const rtm_params* p, const float* d_c, const int32_t* d_rec,
                               float* d_data, const float* d_ae_params, void* d_ws,
                               size_t ws_bytes, rtm_stream stream) {
    CHECK(learned_checks(p, d_c, d_rec, d_ae_params, d_ws, ws_bytes));
    Ctx C;
    CHECK(make_ctx(C, p, d_c, d_ws, stream));
    C.ae = d_ae_params;
    CHECK(run_forward(C, d_rec, d_data, nullptr));
    return finish(C);
}

rtm_status rtm_backward_image_learned(const rtm_params* p, const float* d_c, const int32_t* d_rec,
                                      const float* d_rdata, const float* d_ae_params, void* d_ws,
                                      size_t ws_bytes, float* d_image, rtm_stream stream) {
    CHECK(learned_checks(p, d_c, d_rec, d_ae_params, d_ws, ws_bytes));
    if (!d_rdata && p->nrec > 0) return fail(RTM_ERR_INVALID, "receiver data is NULL");
    if (!d_image) return fail(RTM_ERR_INVALID, "image is NULL");
    Ctx C;
    CHECK(make_ctx(C, p, d_c, d_ws, stream));
    C.ae = d_ae_params;
    CHECK(run_backward(C, d_rec, d_rdata, nullptr, false));
    CU(launch_image_finalize(C.G, C.at(C.L.img), d_image, C.s));
    count_launch();
    return finish(C);
}

rtm_status rtm_shot_learned(const rtm_params* p, const float* d_c, const int32_t* d_rec,
                            const float* d_dobs, const float* d_ae_params, void* d_ws,
                            size_t ws_bytes, float* d_image, rtm_stream stream) {
    CHECK(learned_checks(p, d_c, d_rec, d_ae_params, d_ws, ws_bytes));
    if (!d_dobs && p->nrec > 0) return fail(RTM_ERR_INVALID, "observed data is NULL");
    if (!d_image) return fail(RTM_ERR_INVALID, "image is NULL");
    Ctx C;
    CHECK(make_ctx(C, p, d_c, d_ws, stream));
    C.ae = d_ae_params;
    CHECK(run_forward(C, d_rec, nullptr, nullptr));
    CHECK(run_backward(C, d_rec, d_dobs, nullptr, false));
    CU(launch_image_finalize(C.G, C.at(C.L.img), d_image, C.s));
    count_launch();
    return finish(C);
}

rtm_status rtm_backward_image_illum(const rtm_params* p, const float* d_c, const int32_t* d_rec,
                                    const float* d_rdata, const float* d_ae_params, void* d_ws,
                                    size_t ws_bytes, float* d_image, float* d_illum,
                                    rtm_stream stream) {
    CHECK(common_checks(p, d_c, d_rec, d_ws, ws_bytes));
    if (p->want_grad)
        return fail(RTM_ERR_STATE, "workspace prepared for the gradient (want_grad = 1)");
    if (p->storage == RTM_STORE_LEARNED && !d_ae_params)
        return fail(RTM_ERR_INVALID, "learned storage needs the codec parameters");
    if (!d_rdata && p->nrec > 0) return fail(RTM_ERR_INVALID, "receiver data is NULL");
    if (!d_image || !d_illum) return fail(RTM_ERR_INVALID, "image or illumination is NULL");
    Ctx C;
    CHECK(make_ctx(C, p, d_c, d_ws, stream));
    C.ae = d_ae_params;
    C.illum = d_illum;
    CHECK(run_backward(C, d_rec, d_rdata, nullptr, false));
    CU(launch_image_finalize(C.G, C.at(C.L.img), d_image, C.s));
    count_launch();
    return finish(C);
}

int64_t rtm_revolve_cost(int32_t nstates, int32_t slots) {
    if (nstates < 0 || slots < 0) return -1;
    return revolve_cost(nstates, slots);
}

int32_t rtm_revolve_schedule(int32_t nstates, int32_t slots, int32_t* h_actions,
                             int32_t max_actions) {
    if (nstates < 0 || slots < 0) return -1;
    std::vector<RevolveAction> plan;
    if (!revolve_schedule(nstates, slots, plan)) return -1;
    const int32_t n = (int32_t)plan.size();
    if (h_actions && n <= max_actions)
        for (int32_t i = 0; i < n; i++) {
            h_actions[4 * i] = plan[i].op;
            h_actions[4 * i + 1] = plan[i].a;
            h_actions[4 * i + 2] = plan[i].b;
            h_actions[4 * i + 3] = plan[i].c;
        }
    return n;
}

rtm_status rtm_image_filter(const rtm_params* p, const float* d_image, const float* d_illum,
                            float eps_rel, float* d_normalized, float* d_laplacian, void* d_ws,
                            size_t ws_bytes, rtm_stream stream) {
    // only the model grid, the radius and dx matter here
    if (!p) return fail(RTM_ERR_INVALID, "params is NULL");
    if (p->nx < 1 || p->ny < 1 || p->nz < 1)
        return fail(RTM_ERR_INVALID, "model grid %dx%dx%d must be positive", p->nx, p->ny, p->nz);
    if (p->radius != 4 && p->radius != 8)
        return fail(RTM_ERR_UNSUPPORTED, "stencil radius %d (4 or 8 supported)", p->radius);
    if (!(p->dx > 0.0) || !isfinite(p->dx)) return fail(RTM_ERR_INVALID, "dx must be positive");
    if (!d_image) return fail(RTM_ERR_INVALID, "image is NULL");
    if (d_normalized && (!d_illum || !(eps_rel > 0.f)))
        return fail(RTM_ERR_INVALID, "normalisation needs the illumination and eps_rel > 0");
    if (d_normalized && (!d_ws || ws_bytes < kStatusBytes))
        return fail(RTM_ERR_WORKSPACE, "normalisation needs a workspace (its status block)");
    cudaGetLastError();
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const long long n = (long long)p->nx * p->ny * p->nz;
    if (d_normalized) {
        unsigned int* bits = reinterpret_cast<unsigned int*>(reinterpret_cast<char*>(d_ws) + 32);
        CU(launch_image_normalize(d_image, d_illum, n, bits, eps_rel, d_normalized, s));
        count_launch(2);
    }
    if (d_laplacian) {
        LapWeights w;
        memset(&w, 0, sizeof w);
        w.r = p->radius;
        step_weights(p->radius, p->dx, w.a);
        CU(launch_image_laplacian(d_image, p->nx, p->ny, p->nz, w, d_laplacian, s));
        count_launch();
    }
    return RTM_OK;
}

rtm_status rtm_snapshot(const rtm_params* p, const void* d_ws, size_t ws_bytes, int32_t m,
                        float* d_out, rtm_stream stream) {
    CHECK(validate(p));
    CHECK(check_ws(p, const_cast<void*>(d_ws), ws_bytes));
    if (p->storage != RTM_STORE_ALL || p->want_grad)
        return fail(RTM_ERR_STATE, "snapshots are kept only by store-all imaging workspaces");
    if (m < p->image_every || m > p->nt || m % p->image_every)
        return fail(RTM_ERR_INVALID, "no stored snapshot for step %d", m);
    if (!d_out) return fail(RTM_ERR_INVALID, "output is NULL");
    const Dims d = dims_of(p);
    const Layout L = layout_of(p);
    const char* base = reinterpret_cast<const char*>(d_ws) + L.snap +
                       sizeof(float) * L.snap_elems * (size_t)(m / p->image_every - 1);
    const float* src = reinterpret_cast<const float*>(base) + p->nb;
    CU(cudaMemcpy2DAsync(d_out, sizeof(float) * p->nx, src, sizeof(float) * d.NX,
                         sizeof(float) * p->nx, (size_t)p->nz * p->ny, cudaMemcpyDeviceToDevice,
                         reinterpret_cast<cudaStream_t>(stream)));
    return RTM_OK;
}

rtm_status rtm_misfit(const float* d_data, const float* d_obs, int64_t n, float* d_resid,
                      double* d_J, rtm_stream stream) {
    if (n < 0) return fail(RTM_ERR_INVALID, "n %lld < 0", (long long)n);
    if (!d_J || (n > 0 && (!d_data || !d_obs)))
        return fail(RTM_ERR_INVALID, "misfit arrays are NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CU(cudaMemsetAsync(d_J, 0, sizeof(double), s));
    if (n > 0) {
        CU(launch_misfit(d_data, d_obs, n, d_resid, d_J, s));
        count_launch();
    }
    return RTM_OK;
}

size_t rtm_host_workspace_size(const rtm_params* p) {
    if (validate(p) != RTM_OK) return 0;
    const Dims d = dims_of(p);
    size_t t = layout_of(p).total;
    t += up(sizeof(float) * d.nmodel);             // velocity
    t += up(sizeof(float) * d.N);                  // coefficients
    t += up(sizeof(int32_t) * 3 * (size_t)p->nrec);  // receivers
    t += up(sizeof(float) * (size_t)p->nt * p->nrec);  // data
    t += up(sizeof(float) * d.nmodel);             // image
    return t;
}

rtm_status rtm_shot_host(const rtm_params* p, const float* h_vel, int32_t vel_kind,
                         const int32_t* h_rec, const float* h_dobs, float* h_image, void* d_ws,
                         size_t ws_bytes, rtm_stream stream) {
    CHECK(validate(p));
    if (!h_vel || !h_image || (p->nrec > 0 && (!h_rec || !h_dobs)))
        return fail(RTM_ERR_INVALID, "host array is NULL");
    if (!d_ws) return fail(RTM_ERR_WORKSPACE, "workspace is NULL");
    if ((uintptr_t)d_ws % kAlign) return fail(RTM_ERR_WORKSPACE, "workspace not 256-byte aligned");
    const size_t need = rtm_host_workspace_size(p);
    if (ws_bytes < need)
        return fail(RTM_ERR_WORKSPACE, "workspace %zu bytes, %zu needed", ws_bytes, need);
    const Dims d = dims_of(p);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char* base = reinterpret_cast<char*>(d_ws);
    size_t off = layout_of(p).total;
    float* vel = reinterpret_cast<float*>(base + off);
    off += up(sizeof(float) * d.nmodel);
    float* c = reinterpret_cast<float*>(base + off);
    off += up(sizeof(float) * d.N);
    int32_t* rec = reinterpret_cast<int32_t*>(base + off);
    off += up(sizeof(int32_t) * 3 * (size_t)p->nrec);
    float* dobs = reinterpret_cast<float*>(base + off);
    off += up(sizeof(float) * (size_t)p->nt * p->nrec);
    float* img = reinterpret_cast<float*>(base + off);
    // the observed data are read only by the receiver pass: they travel on a
    // side stream while the model is prepared and the source is propagated.
    // That copy starts after the velocity and receiver uploads: two
    // host-to-device copies at once ran far below the rate of one, and
    // slower with every repetition, while one copy beside the kernels keeps
    // the full rate
    struct Side {
        cudaStream_t st = nullptr;
        cudaEvent_t up = nullptr;  // velocity and receivers uploaded
        cudaEvent_t ev = nullptr;  // observed data uploaded
        ~Side() {
            if (st) cudaStreamSynchronize(st);
            if (ev) cudaEventDestroy(ev);
            if (up) cudaEventDestroy(up);
            if (st) cudaStreamDestroy(st);
        }
    } side;
    CU(cudaStreamCreateWithFlags(&side.st, cudaStreamNonBlocking));
    CU(cudaEventCreateWithFlags(&side.up, cudaEventDisableTiming));
    CU(cudaEventCreateWithFlags(&side.ev, cudaEventDisableTiming));
    CU(cudaMemcpyAsync(vel, h_vel, sizeof(float) * d.nmodel, cudaMemcpyHostToDevice, s));
    if (p->nrec > 0)
        CU(cudaMemcpyAsync(rec, h_rec, sizeof(int32_t) * 3 * (size_t)p->nrec,
                           cudaMemcpyHostToDevice, s));
    CU(cudaEventRecord(side.up, s));
    CU(cudaStreamWaitEvent(side.st, side.up, 0));
    if (p->nrec > 0)
        CU(cudaMemcpyAsync(dobs, h_dobs, sizeof(float) * (size_t)p->nt * p->nrec,
                           cudaMemcpyHostToDevice, side.st));
    CU(cudaEventRecord(side.ev, side.st));
    CHECK(rtm_model_prep(p, vel, vel_kind, c, d_ws, ws_bytes, stream));
    CU(cudaMemsetAsync(img, 0, sizeof(float) * d.nmodel, s));
    CHECK(rtm_forward(p, c, rec, nullptr, d_ws, ws_bytes, nullptr, stream));
    CU(cudaStreamWaitEvent(s, side.ev, 0));
    CHECK(rtm_backward_image(p, c, rec, dobs, d_ws, ws_bytes, img, nullptr, stream));
    CU(cudaMemcpyAsync(h_image, img, sizeof(float) * d.nmodel, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    return RTM_OK;
}

rtm_status rtm_check(void* d_ws, size_t ws_bytes, rtm_stream stream) {
    if (!d_ws || ws_bytes < kStatusBytes) return fail(RTM_ERR_WORKSPACE, "workspace missing");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int h = 0;
    int* st = reinterpret_cast<int*>(d_ws);  // the status word is the first field
    CU(cudaMemcpyAsync(&h, st, sizeof h, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    CU(cudaMemsetAsync(st, 0, sizeof(int), s));
    CU(cudaStreamSynchronize(s));
    if (h == RTM_ERR_INVALID) return fail(RTM_ERR_INVALID, "a receiver lies outside the padded grid");
    if (h == RTM_ERR_TIMEOUT) return fail(RTM_ERR_TIMEOUT, "a bounded device wait ran out");
    if (h == RTM_ERR_NUMERIC)
        return fail(RTM_ERR_NUMERIC, "a wavefield, image or gradient holds non-finite values");
    if (h != 0) return fail((rtm_status)h, "device status %d", h);
    return RTM_OK;
}

rtm_status rtm_set_tuning(int32_t radius, int32_t zchunk, int32_t variant) {
    if (radius != 4 && radius != 8) return fail(RTM_ERR_UNSUPPORTED, "radius %d", radius);
    if (zchunk < 0 || variant < 0 || variant > 3)
        return fail(RTM_ERR_INVALID, "zchunk %d / variant %d out of range", zchunk, variant);
    std::lock_guard<std::mutex> lk(g_mu);
    g_zchunk[radius] = zchunk;
    g_variant[radius] = variant;
    for (int m = 0; m < MODE_COUNT; m++) g_zchunk_mode[radius][m] = 0;
    return RTM_OK;
}

rtm_status rtm_set_test_stall(int32_t kernel, int32_t plane) {
    if (kernel < 0 || kernel >= kStallKernels)
        return (rtm_status)rtm::set_error(RTM_ERR_INVALID, "unknown stall kernel %d", kernel);
    g_test_stall[kernel].store(plane < 0 ? -1 : plane);
    return RTM_OK;
}

rtm_status rtm_set_tuning_mode(int32_t radius, int32_t mode, int32_t zchunk) {
    if (radius != 4 && radius != 8) return fail(RTM_ERR_UNSUPPORTED, "radius %d", radius);
    if (mode < 0 || mode >= MODE_COUNT || mode == 5 || mode == MODE_FWD_SUMSQ || zchunk < 0)
        return fail(RTM_ERR_INVALID, "mode %d / zchunk %d out of range", mode, zchunk);
    std::lock_guard<std::mutex> lk(g_mu);
    g_zchunk_mode[radius][mode] = zchunk;
    return RTM_OK;
}

rtm_status rtm_set_timing(int32_t enable) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_timing = enable != 0;
    return RTM_OK;
}

rtm_status rtm_stats_get(rtm_stats* out) {
    if (!out) return fail(RTM_ERR_INVALID, "stats pointer is NULL");
    std::lock_guard<std::mutex> lk(g_mu);
    *out = g_stats;
    return RTM_OK;
}

rtm_status rtm_stats_reset(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    memset(&g_stats, 0, sizeof g_stats);
    return RTM_OK;
}

}  // extern "C"
