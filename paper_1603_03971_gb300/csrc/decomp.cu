// Single-shot forward modelling on an X-Y domain decomposition of the padded
// grid, with the halo exchange overlapped with the interior stencil.
//
// The paper's distributed time step (Sec. II): apply the stencil to the halo
// regions first, pack them, start the nonblocking exchange with the
// neighbours, apply the stencil to the interior while the messages travel,
// wait, unpack. Its dedicated communication thread (Sec. III) is a
// communication stream here. The subdomains of one call live on one GPU; the
// exchange of a strip is a device copy from the sender's pack buffer into the
// receiver's unpack buffer, the step that a point-to-point message performs
// between GPUs.
//
// Layout. Subdomain s owns padded x in [X0, X1) (X0, X1 multiples of 4, the
// tensor-copy rule) and y in [Y0, Y1), all z. Its fields, coefficients and
// sponge profiles are local arrays of (X1 - X0 + 2r) x (Y1 - Y0 + 2r) x NZ
// cells: the owned block plus an r-wide halo on the four x-y faces. A halo
// facing a neighbour holds that neighbour's owned cells of the newest field;
// a halo on the grid's outer face stays zero (the Dirichlet ghost cells).
// The star stencil reads along the axes only, so the corner blocks of the
// halo are never read and never exchanged.
//
// Each step of subdomain s on its compute stream (up to eight streams, so
// that the subdomains' launches overlap on the GPU as their ranks' would):
// the source pre-adjust and receiver gather (as in the single-domain forward
// pass); the band launches (tiles within 64 columns or 16 rows of a face that
// has a neighbour, which contain every cell the neighbours need); an event;
// the interior launch.
// On the communication stream, after that event: one pack kernel gathers the
// r-wide strips of every subdomain into its send buffer, one copy per face
// moves each strip into the neighbour's receive buffer, one unpack kernel
// scatters the receive buffers into the halos; the next step's band launches
// wait for it. Each launch writes only the cells of its region (the stencil
// kernel bounds its stores by the launch region), so the exchange writing a
// halo and the interior launch writing owned cells never touch the same
// cell, and every cell is computed with the same arithmetic as in the
// single-domain pass: the results equal that pass's bit for bit.

#include <string.h>

#include <algorithm>
#include <vector>

#include "../../include/rtm.h"
#include "rtm_internal.h"

using namespace rtm;

namespace {

constexpr int kBandX = 64;  // band width in x: one tile column (64 or 32 wide)
constexpr int kBandY = 16;  // band height in y: one or two tile rows
constexpr int kMaxSub = 256;
constexpr size_t kAlignD = 256;

size_t upd(size_t v) { return (v + kAlignD - 1) / kAlignD * kAlignD; }

// one r-wide strip of a subdomain's field: packed into (or unpacked from) a
// contiguous buffer, every z plane
struct HaloStrip {
    float* f[2];  // the subdomain's field pair
    float* buf;   // send buffer (pack) or receive buffer (unpack) of the strip
    int x0, y0, w, h;
    int NX, NY, NZ;
};

__global__ void k_halo_copy(const HaloStrip* __restrict__ strips, int which, int unpack) {
    const HaloStrip S = strips[blockIdx.y];
    const long long n = (long long)S.w * S.h * S.NZ;
    const long long plane = (long long)S.w * S.h;
    float* f = S.f[which];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        const int z = (int)(e / plane);
        const int r = (int)(e % plane);
        const int yy = r / S.w, xx = r % S.w;
        float* cell = f + ((long long)z * S.NY + (S.y0 + yy)) * S.NX + S.x0 + xx;
        if (unpack)
            *cell = S.buf[e];
        else
            S.buf[e] = *cell;
    }
}

// data[n][map[j]] = local[n][j] for the receivers of one subdomain
__global__ void k_scatter_traces(const float* __restrict__ local, const int32_t* __restrict__ map,
                                 int m, int nt, int nrec, float* __restrict__ data) {
    const long long n = (long long)nt * m;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        const int t = (int)(e / m), j = (int)(e % m);
        data[(long long)t * nrec + map[j]] = local[e];
    }
}

enum Face { FW = 0, FE = 1, FS = 2, FN = 3 };

struct Sub {
    int X0, X1, Y0, Y1;  // owned range, padded coordinates
    int ox, oy, NXl, NYl;
    int nbr[4];          // neighbour per face (W, E, S, N), -1 at the grid's outer faces
    size_t strip[4];     // floats of the strip sent through each face
    size_t f[2], c, gx, gy, send, recv;  // workspace offsets
    int rec0, nrec;      // receiver slots [rec0, rec0 + nrec) of the pools
    long long src;       // local linear index of the source, or -1
};

struct Plan {
    int px, py, NX, NY, NZ, r;
    std::vector<Sub> sub;
    size_t status, wavelet, gx, gy, gz, strips, rec, map, data, total;
    int nstrips;  // pack (= unpack) descriptors
};

int plan_of(const rtm_params* p, int px, int py, Plan& P) {
    if (rtm_validate(p) != RTM_OK) return RTM_ERR_INVALID;
    if (px < 1 || py < 1 || px * py > kMaxSub)
        return set_error(RTM_ERR_INVALID, "decomposition %d x %d outside 1..%d subdomains", px, py,
                         kMaxSub);
    P.px = px;
    P.py = py;
    P.r = p->radius;
    P.NX = p->nx + 2 * p->nb;
    P.NY = p->ny + 2 * p->nb;
    P.NZ = p->nz + 2 * p->nb;
    const int r = P.r;
    std::vector<int> xb(px + 1), yb(py + 1);
    for (int i = 0; i <= px; i++) xb[i] = (int)((long long)P.NX * i / px / 4 * 4);
    xb[px] = P.NX;
    for (int j = 0; j <= py; j++) yb[j] = (int)((long long)P.NY * j / py);
    for (int i = 0; i < px; i++)
        if (xb[i + 1] - xb[i] < std::max(r, 4))
            return set_error(RTM_ERR_INVALID,
                             "x part %d of %d is %d cells wide: at least r = %d and 4 needed", i,
                             px, xb[i + 1] - xb[i], r);
    for (int j = 0; j < py; j++)
        if (yb[j + 1] - yb[j] < r)
            return set_error(RTM_ERR_INVALID, "y part %d of %d is %d rows: at least r = %d needed",
                             j, py, yb[j + 1] - yb[j], r);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += upd(bytes);
        return o;
    };
    P.status = take(256);
    P.wavelet = take(sizeof(float) * (size_t)p->nt);
    P.gx = take(sizeof(float) * P.NX);
    P.gy = take(sizeof(float) * P.NY);
    P.gz = take(sizeof(float) * P.NZ);
    P.sub.assign((size_t)px * py, Sub{});
    P.nstrips = 0;
    for (int j = 0; j < py; j++)
        for (int i = 0; i < px; i++) {
            Sub& s = P.sub[(size_t)j * px + i];
            s.X0 = xb[i];
            s.X1 = xb[i + 1];
            s.Y0 = yb[j];
            s.Y1 = yb[j + 1];
            s.ox = s.X1 - s.X0;
            s.oy = s.Y1 - s.Y0;
            s.NXl = s.ox + 2 * r;
            s.NYl = s.oy + 2 * r;
            s.nbr[FW] = i > 0 ? j * px + i - 1 : -1;
            s.nbr[FE] = i + 1 < px ? j * px + i + 1 : -1;
            s.nbr[FS] = j > 0 ? (j - 1) * px + i : -1;
            s.nbr[FN] = j + 1 < py ? (j + 1) * px + i : -1;
            s.strip[FW] = s.strip[FE] = (size_t)r * s.oy * P.NZ;
            s.strip[FS] = s.strip[FN] = (size_t)s.ox * r * P.NZ;
            for (int f = 0; f < 4; f++) P.nstrips += s.nbr[f] >= 0;
            const size_t fb = sizeof(float) * (size_t)s.NXl * s.NYl * P.NZ;
            s.f[0] = take(fb);
            s.f[1] = take(fb);
            s.c = take(fb);
            s.gx = take(sizeof(float) * s.NXl);
            s.gy = take(sizeof(float) * s.NYl);
            const size_t sb = sizeof(float) * (s.strip[0] + s.strip[1] + s.strip[2] + s.strip[3]);
            s.send = take(sb);
            s.recv = take(sb);
        }
    P.strips = take(sizeof(HaloStrip) * 2 * (size_t)(P.nstrips ? P.nstrips : 1));
    P.rec = take(sizeof(int32_t) * 3 * (size_t)(p->nrec ? p->nrec : 1));
    P.map = take(sizeof(int32_t) * (size_t)(p->nrec ? p->nrec : 1));
    P.data = take(sizeof(float) * (size_t)p->nt * (size_t)(p->nrec ? p->nrec : 1));
    P.total = off;
    return RTM_OK;
}

size_t strip_offset(const Sub& s, int face) {
    size_t o = 0;
    for (int f = 0; f < face; f++) o += s.strip[f];
    return o;
}

// the strip of face f that s sends (its own cells) or receives (its halo),
// in local coordinates: x0, y0, w, h
void strip_rect(const Sub& s, int r, int face, bool halo, int* q) {
    switch (face) {
        case FW: q[0] = halo ? 0 : r, q[1] = r, q[2] = r, q[3] = s.oy; break;
        case FE: q[0] = halo ? r + s.ox : s.ox, q[1] = r, q[2] = r, q[3] = s.oy; break;
        case FS: q[0] = r, q[1] = halo ? 0 : r, q[2] = s.ox, q[3] = r; break;
        default: q[0] = r, q[1] = halo ? r + s.oy : s.oy, q[2] = s.ox, q[3] = r; break;
    }
}

#define DCU(call)                                                                      \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return (rtm_status)set_error(RTM_ERR_CUDA, "%s failed: %s", #call,          \
                                         cudaGetErrorString(e_));                      \
    } while (0)

constexpr int kMaxStreams = 8;  // compute streams; subdomain k runs on stream k % n

// the compute streams (subdomains' launches overlap, as their ranks' would),
// the communication stream and their events, owned by one call
struct Streams {
    int n = 0;
    cudaStream_t comp[kMaxStreams] = {nullptr};
    cudaEvent_t band[kMaxStreams] = {nullptr};  // a compute stream's band launches are done
    cudaStream_t comm = nullptr;
    cudaEvent_t start = nullptr, done = nullptr;  // set-up done; a step's exchange done
    ~Streams() {
        for (int i = 0; i < n; i++) {
            if (band[i]) cudaEventDestroy(band[i]);
            if (comp[i]) cudaStreamDestroy(comp[i]);
        }
        if (done) cudaEventDestroy(done);
        if (start) cudaEventDestroy(start);
        if (comm) cudaStreamDestroy(comm);
    }
};

}  // namespace

extern "C" {

int32_t rtm_decomp_plan(const rtm_params* p, int32_t px, int32_t py, int32_t* h_out,
                        int32_t max_sub) {
    Plan P;
    if (plan_of(p, px, py, P) != RTM_OK) return -1;
    const int n = px * py;
    if (h_out && n <= max_sub)
        for (int k = 0; k < n; k++) {
            const Sub& s = P.sub[k];
            int32_t* o = h_out + 8 * k;
            o[0] = s.X0, o[1] = s.X1, o[2] = s.Y0, o[3] = s.Y1;
            for (int f = 0; f < 4; f++) o[4 + f] = s.nbr[f];
        }
    return n;
}

size_t rtm_decomp_workspace_size(const rtm_params* p, int32_t px, int32_t py) {
    Plan P;
    if (plan_of(p, px, py, P) != RTM_OK) return 0;
    return P.total;
}

rtm_status rtm_forward_decomposed(const rtm_params* p, int32_t px, int32_t py, const float* d_c,
                                  const int32_t* d_rec, float* d_data, void* d_ws,
                                  size_t ws_bytes, float* d_u_last, rtm_stream stream) {
    Plan P;
    int st = plan_of(p, px, py, P);
    if (st != RTM_OK) return (rtm_status)st;
    if (p->storage != RTM_STORE_ALL && p->storage != RTM_STORE_CKPT)
        return (rtm_status)set_error(RTM_ERR_INVALID,
                                     "the decomposed forward pass models data only: storage must "
                                     "be RTM_STORE_ALL or RTM_STORE_CKPT (nothing is stored)");
    if (p->want_grad)
        return (rtm_status)set_error(RTM_ERR_INVALID, "the decomposed forward pass models data only");
    if (!d_c || (uintptr_t)d_c % 16)
        return (rtm_status)set_error(RTM_ERR_INVALID, "coefficient grid NULL or not 16-byte aligned");
    if (p->nrec > 0 && !d_rec)
        return (rtm_status)set_error(RTM_ERR_INVALID, "receiver array is NULL");
    if (!d_ws || (uintptr_t)d_ws % kAlignD)
        return (rtm_status)set_error(RTM_ERR_WORKSPACE, "workspace NULL or not 256-byte aligned");
    if (ws_bytes < P.total)
        return (rtm_status)set_error(RTM_ERR_WORKSPACE, "workspace %zu bytes, %zu needed", ws_bytes,
                                     P.total);
    if (!tma_available())
        return (rtm_status)set_error(RTM_ERR_UNSUPPORTED,
                                     "the decomposed pass needs the TMA stencil (tensor maps)");
    cudaGetLastError();
    cudaStream_t S = reinterpret_cast<cudaStream_t>(stream);
    char* ws = reinterpret_cast<char*>(d_ws);
    auto F = [&](size_t off) { return reinterpret_cast<float*>(ws + off); };
    const int r = P.r, NZ = P.NZ, NX = P.NX, NY = P.NY;
    const int nsub = px * py;
    int* status = reinterpret_cast<int*>(ws + P.status);

    // ---- receivers and source: owner subdomains and local coordinates (host)
    std::vector<int32_t> rec((size_t)3 * p->nrec);
    if (p->nrec > 0)
        DCU(cudaMemcpy(rec.data(), d_rec, sizeof(int32_t) * rec.size(), cudaMemcpyDeviceToHost));
    auto owner = [&](int xg, int yg, int zg) -> int {
        if (xg < 0 || xg >= NX || yg < 0 || yg >= NY || zg < 0 || zg >= NZ) return -1;
        int i = 0, j = 0;
        while (i + 1 < px && xg >= P.sub[i + 1].X0) i++;
        while (j + 1 < py && yg >= P.sub[(size_t)(j + 1) * px].Y0) j++;
        return j * px + i;
    };
    std::vector<std::vector<int>> mine(nsub);
    bool outside = false;
    for (int j = 0; j < p->nrec; j++) {
        const int o = owner(rec[3 * j] + p->nb, rec[3 * j + 1] + p->nb, rec[3 * j + 2] + p->nb);
        if (o < 0)
            outside = true;
        else
            mine[o].push_back(j);
    }
    std::vector<int32_t> lrec, lmap;
    for (int k = 0; k < nsub; k++) {
        Sub& s = P.sub[k];
        s.rec0 = (int)lmap.size();
        s.nrec = (int)mine[k].size();
        for (int j : mine[k]) {
            // model coordinates whose padded position is the local one
            lrec.push_back(rec[3 * j] + p->nb - s.X0 + r - p->nb);
            lrec.push_back(rec[3 * j + 1] + p->nb - s.Y0 + r - p->nb);
            lrec.push_back(rec[3 * j + 2]);
            lmap.push_back(j);
        }
        s.src = -1;
    }
    const int sxg = p->src_x + p->nb, syg = p->src_y + p->nb, szg = p->src_z + p->nb;
    const int so = owner(sxg, syg, szg);
    {
        Sub& s = P.sub[so];
        s.src = ((long long)szg * s.NYl + (syg - s.Y0 + r)) * s.NXl + (sxg - s.X0 + r);
    }

    // ---- halo strip descriptors: pack (send) and unpack (receive)
    std::vector<HaloStrip> hs;
    for (int pass = 0; pass < 2; pass++)
        for (int k = 0; k < nsub; k++) {
            const Sub& s = P.sub[k];
            for (int f = 0; f < 4; f++) {
                if (s.nbr[f] < 0) continue;
                HaloStrip h;
                int q[4];
                strip_rect(s, r, f, pass == 1, q);
                h.f[0] = F(s.f[0]);
                h.f[1] = F(s.f[1]);
                h.buf = F(pass == 0 ? s.send : s.recv) + strip_offset(s, f);
                h.x0 = q[0], h.y0 = q[1], h.w = q[2], h.h = q[3];
                h.NX = s.NXl, h.NY = s.NYl, h.NZ = NZ;
                hs.push_back(h);
            }
        }
    HaloStrip* d_strips = reinterpret_cast<HaloStrip*>(ws + P.strips);
    if (!hs.empty())
        DCU(cudaMemcpyAsync(d_strips, hs.data(), sizeof(HaloStrip) * hs.size(),
                            cudaMemcpyHostToDevice, S));
    int32_t* d_lrec = reinterpret_cast<int32_t*>(ws + P.rec);
    int32_t* d_lmap = reinterpret_cast<int32_t*>(ws + P.map);
    if (!lmap.empty()) {
        DCU(cudaMemcpyAsync(d_lrec, lrec.data(), sizeof(int32_t) * lrec.size(),
                            cudaMemcpyHostToDevice, S));
        DCU(cudaMemcpyAsync(d_lmap, lmap.data(), sizeof(int32_t) * lmap.size(),
                            cudaMemcpyHostToDevice, S));
    }
    // the host vectors must outlive the copies
    DCU(cudaStreamSynchronize(S));

    // ---- tables, local coefficients and profiles, zero fields
    DCU(cudaMemsetAsync(status, 0, sizeof(int), S));
    const Geometry G{NX, NY, NZ, p->nb, p->nx, p->ny, p->nz};
    DCU(launch_wavelet(p->nt, p->dt, p->f0, p->t0, F(P.wavelet), S));
    DCU(launch_sponge(G, F(P.gx), F(P.gy), F(P.gz), S));
    static const int kInvalid = RTM_ERR_INVALID;
    if (outside)  // a receiver outside the padded grid: no trace, status word set
        DCU(cudaMemcpyAsync(status, &kInvalid, sizeof(int), cudaMemcpyHostToDevice, S));
    for (int k = 0; k < nsub; k++) {
        const Sub& s = P.sub[k];
        const size_t fb = sizeof(float) * (size_t)s.NXl * s.NYl * NZ;
        DCU(cudaMemsetAsync(F(s.f[0]), 0, fb, S));
        DCU(cudaMemsetAsync(F(s.f[1]), 0, fb, S));
        DCU(cudaMemsetAsync(F(s.c), 0, fb, S));
        DCU(cudaMemsetAsync(F(s.gx), 0, sizeof(float) * s.NXl, S));
        DCU(cudaMemsetAsync(F(s.gy), 0, sizeof(float) * s.NYl, S));
        // the owned block and the halo inside the padded grid
        const int gx0 = std::max(s.X0 - r, 0), gx1 = std::min(s.X1 + r, NX);
        const int gy0 = std::max(s.Y0 - r, 0), gy1 = std::min(s.Y1 + r, NY);
        cudaMemcpy3DParms m;
        memset(&m, 0, sizeof m);
        m.srcPtr = make_cudaPitchedPtr(const_cast<float*>(d_c), sizeof(float) * NX, NX, NY);
        m.srcPos = make_cudaPos(sizeof(float) * gx0, gy0, 0);
        m.dstPtr = make_cudaPitchedPtr(F(s.c), sizeof(float) * s.NXl, s.NXl, s.NYl);
        m.dstPos = make_cudaPos(sizeof(float) * (gx0 - s.X0 + r), gy0 - s.Y0 + r, 0);
        m.extent = make_cudaExtent(sizeof(float) * (gx1 - gx0), gy1 - gy0, NZ);
        m.kind = cudaMemcpyDeviceToDevice;
        DCU(cudaMemcpy3DAsync(&m, S));
        DCU(cudaMemcpyAsync(F(s.gx) + (gx0 - s.X0 + r), F(P.gx) + gx0,
                            sizeof(float) * (gx1 - gx0), cudaMemcpyDeviceToDevice, S));
        DCU(cudaMemcpyAsync(F(s.gy) + (gy0 - s.Y0 + r), F(P.gy) + gy0,
                            sizeof(float) * (gy1 - gy0), cudaMemcpyDeviceToDevice, S));
    }

    // ---- launch shapes
    const int var = tuning_variant(r);
    const int tile_rows = var == 2 ? 16 : 8;
    const int zc_set = tuning_zchunk(r);
    std::vector<StepArgs> base(nsub);
    for (int k = 0; k < nsub; k++) {
        const Sub& s = P.sub[k];
        StepArgs& a = base[k];
        memset(&a, 0, sizeof a);
        step_weights(r, p->dx, a.a);
        a.c = F(s.c);
        a.gx = F(s.gx);
        a.gy = F(s.gy);
        a.gz = F(P.gz);
        a.NX = s.NXl;
        a.NY = s.NYl;
        a.NZ = NZ;
        a.nb = p->nb;
        a.nx = p->nx;
        a.ny = p->ny;
        a.nz = p->nz;
        a.zchunk = zc_set > 0 ? zc_set : auto_zchunk(r, s.ox, s.oy, NZ);
        if ((NZ + a.zchunk - 1) / a.zchunk > 65535) a.zchunk = (NZ + 65534) / 65535;
        a.zorg = 0;
        a.zend = NZ;
    }
    // regions [x0, x1) x [y0, y1) of the band launches and of the interior
    struct Rect {
        int x0, x1, y0, y1;
    };
    std::vector<std::vector<Rect>> band(nsub);
    std::vector<Rect> inner(nsub);
    for (int k = 0; k < nsub; k++) {
        const Sub& s = P.sub[k];
        const int bl = s.nbr[FW] >= 0 ? std::min(kBandX, s.ox) : 0;
        const int br = s.nbr[FE] >= 0 ? std::min(kBandX, s.ox - bl) : 0;
        const int bs = s.nbr[FS] >= 0 ? std::min(kBandY, s.oy) : 0;
        const int bn = s.nbr[FN] >= 0 ? std::min(kBandY, s.oy - bs) : 0;
        const int xl = r + bl, xr = r + s.ox - br, yl = r + bs, yr = r + s.oy - bn;
        if (bl > 0) band[k].push_back({r, r + bl, r, r + s.oy});
        if (br > 0) band[k].push_back({r + s.ox - br, r + s.ox, r, r + s.oy});
        if (bs > 0 && xr > xl) band[k].push_back({xl, xr, r, r + bs});
        if (bn > 0 && xr > xl) band[k].push_back({xl, xr, r + s.oy - bn, r + s.oy});
        inner[k] = {xl, xr, yl, yr};
    }
    Streams C;
    C.n = std::min(nsub, kMaxStreams);
    for (int i = 0; i < C.n; i++) {
        DCU(cudaStreamCreateWithFlags(&C.comp[i], cudaStreamNonBlocking));
        DCU(cudaEventCreateWithFlags(&C.band[i], cudaEventDisableTiming));
    }
    DCU(cudaStreamCreateWithFlags(&C.comm, cudaStreamNonBlocking));
    DCU(cudaEventCreateWithFlags(&C.start, cudaEventDisableTiming));
    DCU(cudaEventCreateWithFlags(&C.done, cudaEventDisableTiming));
    DCU(cudaEventRecord(C.start, S));  // the set-up above
    for (int i = 0; i < C.n; i++) DCU(cudaStreamWaitEvent(C.comp[i], C.start, 0));
    DCU(cudaStreamWaitEvent(C.comm, C.start, 0));
    auto stream_of = [&](int k) { return C.comp[k % C.n]; };
    auto launch = [&](int k, const Rect& q, float* cur, float* prev) -> cudaError_t {
        if (q.x1 <= q.x0 || q.y1 <= q.y0) return cudaSuccess;
        StepArgs a = base[k];
        a.u_cur = cur;
        a.u_prev = prev;
        a.xorg = q.x0;
        a.xend = q.x1;
        a.yorg = q.y0;
        a.yend = q.y1;
        return launch_stencil_tma(r, MODE_FWD, a, status, stream_of(k), tile_rows);
    };
    const int npack = (int)hs.size() / 2;
    size_t max_strip = 1;
    for (const HaloStrip& h : hs) max_strip = std::max(max_strip, (size_t)h.w * h.h * h.NZ);
    const int gx_blocks = (int)std::min<size_t>((max_strip + 255) / 256, 152 * 4);
    const float inv_dx3 = (float)(1.0 / (p->dx * p->dx * p->dx));
    float* ldata = F(P.data);

    // ---- the time loop
    for (int n = 0; n < p->nt; n++) {
        const int wn = n % 2;  // the new field u^{n+1} lands in f[wn]
        if (n > 0)  // halos of u^n are in
            for (int i = 0; i < C.n; i++) DCU(cudaStreamWaitEvent(C.comp[i], C.done, 0));
        for (int k = 0; k < nsub; k++) {
            const Sub& s = P.sub[k];
            if (s.nrec == 0 && s.src < 0) continue;
            const Geometry Gl{s.NXl, s.NYl, NZ, p->nb, p->nx, p->ny, p->nz};
            float* row = (d_data && n >= 1 && s.nrec > 0)
                             ? ldata + (size_t)p->nt * s.rec0 + (size_t)(n - 1) * s.nrec
                             : nullptr;
            DCU(launch_fwd_aux(Gl, F(s.f[1 - wn]), F(s.f[wn]), F(s.c), F(s.gx), F(s.gy),
                               F(P.gz), d_lrec + 3 * (size_t)s.rec0, s.nrec, row,
                               s.src >= 0 ? s.src : 0, s.src >= 0 ? F(P.wavelet) + n : nullptr,
                               inv_dx3, status, stream_of(k)));
        }
        for (int k = 0; k < nsub; k++)
            for (const Rect& q : band[k]) DCU(launch(k, q, F(P.sub[k].f[1 - wn]), F(P.sub[k].f[wn])));
        for (int i = 0; i < C.n; i++) {
            DCU(cudaEventRecord(C.band[i], C.comp[i]));
            DCU(cudaStreamWaitEvent(C.comm, C.band[i], 0));
        }
        if (npack > 0) {
            k_halo_copy<<<dim3(gx_blocks, npack), 256, 0, C.comm>>>(d_strips, wn, 0);
            DCU(cudaGetLastError());
            for (int k = 0; k < nsub; k++) {
                const Sub& s = P.sub[k];
                for (int f = 0; f < 4; f++) {
                    const int t = s.nbr[f];
                    if (t < 0) continue;
                    const Sub& d = P.sub[t];
                    const int g = f ^ 1;  // the face of t that looks back at s
                    DCU(cudaMemcpyAsync(F(d.recv) + strip_offset(d, g), F(s.send) + strip_offset(s, f),
                                        sizeof(float) * s.strip[f], cudaMemcpyDeviceToDevice,
                                        C.comm));
                }
            }
            k_halo_copy<<<dim3(gx_blocks, npack), 256, 0, C.comm>>>(d_strips + npack, wn, 1);
            DCU(cudaGetLastError());
        }
        DCU(cudaEventRecord(C.done, C.comm));
        for (int k = 0; k < nsub; k++)
            DCU(launch(k, inner[k], F(P.sub[k].f[1 - wn]), F(P.sub[k].f[wn])));
    }
    // the caller's stream continues after every compute stream and the last exchange
    for (int i = 0; i < C.n; i++) {
        DCU(cudaEventRecord(C.band[i], C.comp[i]));
        DCU(cudaStreamWaitEvent(S, C.band[i], 0));
    }
    DCU(cudaStreamWaitEvent(S, C.done, 0));
    // u^{nt} is in f[(nt - 1) % 2], u^{nt - 1} in f[nt % 2]
    const int last = (p->nt - 1) % 2;
    for (int k = 0; k < nsub; k++) {
        const Sub& s = P.sub[k];
        if (d_data && s.nrec > 0) {
            const Geometry Gl{s.NXl, s.NYl, NZ, p->nb, p->nx, p->ny, p->nz};
            DCU(launch_fwd_aux(Gl, F(s.f[last]), F(s.f[1 - last]), F(s.c), F(s.gx), F(s.gy),
                               F(P.gz), d_lrec + 3 * (size_t)s.rec0, s.nrec,
                               ldata + (size_t)p->nt * s.rec0 + (size_t)(p->nt - 1) * s.nrec, 0,
                               nullptr, inv_dx3, status, S));
        }
        DCU(launch_finite_scan(F(s.f[last]), (long long)s.NXl * s.NYl * NZ, status, S));
    }
    if (d_data && p->nrec > 0) {
        if (outside) DCU(cudaMemsetAsync(d_data, 0, sizeof(float) * (size_t)p->nt * p->nrec, S));
        for (int k = 0; k < nsub; k++) {
            const Sub& s = P.sub[k];
            if (s.nrec == 0) continue;
            const long long n = (long long)p->nt * s.nrec;
            const int blocks = (int)std::min<long long>((n + 255) / 256, 152 * 8);
            k_scatter_traces<<<blocks, 256, 0, S>>>(ldata + (size_t)p->nt * s.rec0,
                                                    d_lmap + s.rec0, s.nrec, p->nt, p->nrec,
                                                    d_data);
            DCU(cudaGetLastError());
        }
    }
    if (d_u_last) {
        const size_t N = (size_t)NX * NY * NZ;
        for (int which = 0; which < 2; which++) {
            // u_last[0] = u^{nt-1}, u_last[1] = u^{nt}
            const int src_f = which == 0 ? 1 - last : last;
            for (int k = 0; k < nsub; k++) {
                const Sub& s = P.sub[k];
                cudaMemcpy3DParms m;
                memset(&m, 0, sizeof m);
                m.srcPtr = make_cudaPitchedPtr(F(s.f[src_f]), sizeof(float) * s.NXl, s.NXl, s.NYl);
                m.srcPos = make_cudaPos(sizeof(float) * r, r, 0);
                m.dstPtr = make_cudaPitchedPtr(d_u_last + which * N, sizeof(float) * NX, NX, NY);
                m.dstPos = make_cudaPos(sizeof(float) * s.X0, s.Y0, 0);
                m.extent = make_cudaExtent(sizeof(float) * s.ox, s.oy, NZ);
                m.kind = cudaMemcpyDeviceToDevice;
                DCU(cudaMemcpy3DAsync(&m, S));
            }
        }
    }
    return RTM_OK;
}

}  // extern "C"
