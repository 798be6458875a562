// C ABI of the batched multi-shot RTM: wave planning under a memory budget,
// per-shot buffers, the common phase schedule, and one CUDA graph per call
// holding every wave's model preparation, persistent launch and image stack.

#include <math.h>
#include <string.h>

#include <algorithm>
#include <memory>
#include <vector>

#include "../../include/rtm.h"
#include "batch_internal.h"

using namespace rtm;

namespace {

constexpr size_t kAlB = 256;
// automatic z-slab height of a work item, per wave: the tallest slab (the
// whole column first) that still gives every phase step at least
// kItemsPerBlock items per resident block. Each step of a shot waits for all
// items of its previous step, so too few items leave blocks idle at every
// step; too short slabs repeat the 2r-plane queue warm-up. Measured with the
// TMA kernel: 4 shots of 256 x 256 x 320 padded, whole columns / 256 / 128
// planes: 137 / 174 / 270 Gpoint-updates/s (radius 4); the 32-shot radius-8
// workload: whole columns 173.8, 128 planes 167.4
constexpr int kBatchZchunk = 128;  // the workspace's sizing value
constexpr int kItemsPerBlock = 3;

int wave_zchunk(const std::vector<BatchShot>& shots, int first, int last, int grid) {
    int nzmax = 1;
    for (int i = first; i < last; i++) nzmax = std::max(nzmax, shots[i].NZ);
    const int cand[] = {nzmax, 512, 384, 256, 192, 128, 96, 64};
    int best = 64;
    for (int zc : cand) {
        if (zc > nzmax) continue;
        long long items = 0;
        for (int i = first; i < last; i++)
            items += (long long)shots[i].tiles_x * shots[i].tiles_y *
                     ((shots[i].NZ + zc - 1) / zc);
        if (items >= (long long)kItemsPerBlock * grid) return zc;
        best = zc;
    }
    return best;
}
double g_wait_seconds = 20.0;  // bound of each inter-block wait
int g_poison_shot = -1;
constexpr int kMaxShotsTotal = 1024;
size_t upb(size_t v) { return (v + kAlB - 1) / kAlB * kAlB; }

#define CUB(call)                                                                       \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return (rtm_status)set_error(RTM_ERR_CUDA, "%s failed: %s", #call,          \
                                         cudaGetErrorString(e_));                       \
    } while (0)

struct Plan {
    std::vector<BatchShot> shots;     // pointers filled per wave
    std::vector<size_t> bytes;        // per-shot buffer bytes
    std::vector<size_t> data_off;     // offset (floats) of each shot's data
    std::vector<std::pair<int, int>> waves;  // [first, last) shots
    std::vector<BatchPhase> phases;
    size_t pool = 0;                  // largest wave
    size_t off_ctrl, off_phases, off_desc, off_wav, off_pool, total;
};

rtm_status check_batch(const rtm_params* p, int nshots, const rtm_aperture* sh) {
    rtm_params q = *p;
    q.storage = RTM_STORE_CKPT;
    q.src_x = q.src_y = q.src_z = 0;
    q.want_grad = 0;
    q.nb = 0;  // the full model itself is not padded
    q.nx += (4 - q.nx % 4) % 4;  // only the apertures' rows must be 16-byte aligned
    rtm_status st = rtm_validate(&q);
    if (st != RTM_OK) return st;
    if (p->storage != RTM_STORE_CKPT || p->ckpt_every < 1)
        return (rtm_status)set_error(RTM_ERR_INVALID, "the batch checkpoints: storage must be "
                                                      "RTM_STORE_CKPT with ckpt_every >= 1");
    if (nshots < 1 || nshots > kMaxShotsTotal || !sh)
        return (rtm_status)set_error(RTM_ERR_INVALID, "nshots %d out of [1, %d]", nshots,
                                     kMaxShotsTotal);
    for (int s = 0; s < nshots; s++) {
        const rtm_aperture& a = sh[s];
        if (a.nx < 1 || a.ny < 1 || a.nz < 1 || a.ox < 0 || a.oy < 0 || a.oz < 0 ||
            a.ox + a.nx > p->nx || a.oy + a.ny > p->ny || a.oz + a.nz > p->nz)
            return (rtm_status)set_error(RTM_ERR_INVALID, "aperture %d outside the model", s);
        if ((a.nx + 2 * p->nb) % 4)
            return (rtm_status)set_error(RTM_ERR_INVALID,
                                         "aperture %d: nx + 2 nb must be a multiple of 4", s);
        if (a.src_x < 0 || a.src_x >= a.nx || a.src_y < 0 || a.src_y >= a.ny || a.src_z < 0 ||
            a.src_z >= a.nz || a.rec_z < 0 || a.rec_z >= a.nz)
            return (rtm_status)set_error(RTM_ERR_INVALID, "aperture %d: source or receiver "
                                                          "plane outside the aperture", s);
    }
    return RTM_OK;
}

// the batched kernel: TMA plane loads wherever the driver provides tensor maps
// (unless the vector-load variant is selected for the radius)
bool batch_uses_tma(int radius) { return tma_available() && tuning_variant(radius) != 1; }
// tile rows of the TMA kernel: 8 when the 8-row tile (variant 3) is selected
int batch_tile_rows(int radius) { return tuning_variant(radius) == 3 ? 8 : 16; }

Plan make_plan(const rtm_params* p, int nshots, const rtm_aperture* sh, size_t budget,
               int zchunk) {
    const bool tma = batch_uses_tma(p->radius);
    const int tile_y = tma ? batch_tile_rows(p->radius) : 16;
    const int tile_x = tma ? batch_tma_tile_x(p->radius, tile_y) : 64;
    Plan P;
    const int R = p->radius, k = p->ckpt_every, nt = p->nt;
    const int nseg = (nt + k - 1) / k;
    size_t doff = 0;
    for (int s = 0; s < nshots; s++) {
        BatchShot b;
        memset(&b, 0, sizeof b);
        b.nb = p->nb;
        b.nx = sh[s].nx;
        b.ny = sh[s].ny;
        b.nz = sh[s].nz;
        b.NX = b.nx + 2 * p->nb;
        b.NY = b.ny + 2 * p->nb;
        b.NZ = b.nz + 2 * p->nb;
        b.tiles_x = (b.NX + tile_x - 1) / tile_x;
        b.tiles_y = (b.NY + tile_y - 1) / tile_y;
        b.tiles_z = (b.NZ + zchunk - 1) / zchunk;
        b.ntiles = b.tiles_x * b.tiles_y * b.tiles_z;
        b.src_x = sh[s].src_x + p->nb;
        b.src_y = sh[s].src_y + p->nb;
        b.src_z = sh[s].src_z + p->nb;
        b.rec_z = sh[s].rec_z + p->nb;
        const size_t N = (size_t)b.NX * b.NY * b.NZ;
        const size_t slab = (size_t)b.nz * b.ny * b.NX;
        size_t bytes = upb(4 * (size_t)b.NX) + upb(4 * (size_t)b.NY) + upb(4 * (size_t)b.NZ);
        // c, two field pairs and the checkpoints, one stride apart
        bytes += upb(4 * N) * (5 + 2 * (size_t)(nseg > 1 ? nseg - 1 : 0));
        bytes += upb(4 * slab) * ((size_t)k + 1);  // snapshots and the image slab
        P.shots.push_back(b);
        P.bytes.push_back(bytes);
        P.data_off.push_back(doff);
        doff += (size_t)nt * b.nx * b.ny;
        (void)R;
    }
    // waves: consecutive shots while the budget holds (a shot over budget alone)
    int first = 0;
    size_t acc = 0;
    for (int s = 0; s < nshots; s++) {
        const bool full = (s - first) >= kMaxBatchShots;
        if (s > first && (full || (budget && acc + P.bytes[s] > budget))) {
            P.waves.push_back({first, s});
            P.pool = std::max(P.pool, acc);
            first = s;
            acc = 0;
        }
        acc += P.bytes[s];
    }
    P.waves.push_back({first, nshots});
    P.pool = std::max(P.pool, acc);
    // phase schedule
    for (int n = 0; n < nt; n++) P.phases.push_back({PH_FWD, n, 0, 0});
    for (int j = nseg - 1; j >= 0; j--) {
        const int n0 = j * k, n1 = std::min(nt, n0 + k);
        for (int n = n0; n < n1; n++) P.phases.push_back({PH_REC, n, j, n - n0});
        for (int m = n1; m > n0; m--) P.phases.push_back({PH_BWD, m, j, m - 1 - n0});
    }
    size_t off = kAlB;  // status block
    P.off_ctrl = off;
    off += upb(sizeof(BatchCtrl));
    P.off_phases = off;
    off += upb(sizeof(BatchPhase) * P.phases.size());
    P.off_desc = off;
    off += upb(sizeof(BatchShot) * (size_t)nshots);
    P.off_wav = off;
    off += upb(sizeof(float) * (size_t)nt);
    P.off_pool = off;
    off += P.pool;
    P.total = off;
    return P;
}

}  // namespace

extern "C" {

rtm_status rtm_batch_set_wait(double seconds, int32_t poison_shot) {
    if (!(seconds > 0.0) || seconds > 3600.0)
        return (rtm_status)set_error(RTM_ERR_INVALID, "wait bound %g s out of (0, 3600]", seconds);
    g_wait_seconds = seconds;
    g_poison_shot = poison_shot;
    return RTM_OK;
}

size_t rtm_batch_workspace_size(const rtm_params* p, int32_t nshots, const rtm_aperture* h_shots,
                                size_t budget_bytes) {
    if (!p || check_batch(p, nshots, h_shots) != RTM_OK) return 0;
    return make_plan(p, nshots, h_shots, budget_bytes, kBatchZchunk)
        .total;
}

rtm_status rtm_batch(const rtm_params* p, int32_t nshots, const rtm_aperture* h_shots,
                     const float* d_vel, const float* d_dobs, float* d_data, float* d_image,
                     void* d_ws, size_t ws_bytes, size_t budget_bytes, int32_t zchunk,
                     rtm_stream stream) {
    if (!p) return (rtm_status)set_error(RTM_ERR_INVALID, "params is NULL");
    rtm_status st = check_batch(p, nshots, h_shots);
    if (st != RTM_OK) return st;
    if (!d_vel || !d_dobs || !d_image)
        return (rtm_status)set_error(RTM_ERR_INVALID, "batch arrays are NULL");
    if (zchunk < 0) return (rtm_status)set_error(RTM_ERR_INVALID, "zchunk < 0");
    Plan P = make_plan(p, nshots, h_shots, budget_bytes, kBatchZchunk);
    if (!d_ws || ((uintptr_t)d_ws % kAlB))
        return (rtm_status)set_error(RTM_ERR_WORKSPACE, "workspace NULL or not 256-byte aligned");
    if (ws_bytes < P.total)
        return (rtm_status)set_error(RTM_ERR_WORKSPACE, "batch workspace %zu bytes, %zu needed",
                                     ws_bytes, P.total);
    for (auto& w : P.waves)
        if (w.second - w.first > kMaxBatchShots)
            return (rtm_status)set_error(RTM_ERR_INVALID, "wave too large");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char* ws = reinterpret_cast<char*>(d_ws);
    cudaGetLastError();  // a stale error of earlier work must not be taken for ours
    int dev = 0, nsm = 0;
    CUB(cudaGetDevice(&dev));
    CUB(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const bool tma = batch_uses_tma(p->radius);
    const int rows = batch_tile_rows(p->radius);
    const int bps = tma ? batch_tma_blocks_per_sm(p->radius, rows) : batch_blocks_per_sm(p->radius);
    if (bps < 1) return (rtm_status)set_error(RTM_ERR_CUDA, "batch kernel does not fit on an SM");
    int clock_khz = 0;
    CUB(cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, dev));
    // slab height per wave (only the tile counts depend on it)
    std::vector<int> wave_zc;
    for (auto& w : P.waves) {
        const int zc = zchunk > 0 ? zchunk : wave_zchunk(P.shots, w.first, w.second, nsm * bps);
        wave_zc.push_back(zc);
        for (int i = w.first; i < w.second; i++) {
            BatchShot& b = P.shots[i];
            b.tiles_z = (b.NZ + zc - 1) / zc;
            b.ntiles = b.tiles_x * b.tiles_y * b.tiles_z;
        }
    }

    // per-wave buffer pointers and descriptors (all waves share the pool)
    for (auto& w : P.waves) {
        char* q = ws + P.off_pool;
        long long base = 0;
        for (int i = w.first; i < w.second; i++) {
            BatchShot& b = P.shots[i];
            const size_t N = (size_t)b.NX * b.NY * b.NZ;
            const size_t slab = (size_t)b.nz * b.ny * b.NX;
            const int nseg = (p->nt + p->ckpt_every - 1) / p->ckpt_every;
            auto take = [&](size_t bytes) {
                char* r = q;
                q += upb(bytes);
                return reinterpret_cast<float*>(r);
            };
            b.gx = take(4 * (size_t)b.NX);
            b.gy = take(4 * (size_t)b.NY);
            b.gz = take(4 * (size_t)b.NZ);
            b.fstride = (long long)(upb(4 * N) / 4);
            b.c = take(upb(4 * N) * (5 + 2 * (size_t)(nseg > 1 ? nseg - 1 : 0)));
            b.f0 = const_cast<float*>(b.c) + 1 * b.fstride;
            b.f1 = const_cast<float*>(b.c) + 2 * b.fstride;
            b.m0 = const_cast<float*>(b.c) + 3 * b.fstride;
            b.m1 = const_cast<float*>(b.c) + 4 * b.fstride;
            b.ckpt = const_cast<float*>(b.c) + 5 * b.fstride;
            b.sstride = (long long)(upb(4 * slab) / 4);
            b.snap = take(upb(4 * slab) * ((size_t)p->ckpt_every + 1));
            b.img = b.snap + (size_t)p->ckpt_every * b.sstride;
            b.dobs = d_dobs + P.data_off[i];
            b.data = d_data ? d_data + P.data_off[i] : nullptr;
            b.item_base = base;
            base += b.ntiles;
        }
    }
    // static tables (before capture: host sources stay valid until the sync)
    CUB(cudaMemcpyAsync(ws + P.off_phases, P.phases.data(), sizeof(BatchPhase) * P.phases.size(),
                        cudaMemcpyHostToDevice, s));
    CUB(cudaMemcpyAsync(ws + P.off_desc, P.shots.data(), sizeof(BatchShot) * P.shots.size(),
                        cudaMemcpyHostToDevice, s));
    CUB(cudaMemsetAsync(ws, 0, sizeof(int), s));
    CUB(launch_wavelet(p->nt, p->dt, p->f0, p->t0, reinterpret_cast<float*>(ws + P.off_wav), s));
    CUB(cudaStreamSynchronize(s));

    BatchArgs A;
    memset(&A, 0, sizeof A);
    std::unique_ptr<BatchTmaArgs> T(tma ? new BatchTmaArgs() : nullptr);
    step_weights(p->radius, p->dx, A.a);
    A.inv_dx3 = (float)(1.0 / (p->dx * p->dx * p->dx));
    A.phases = reinterpret_cast<const BatchPhase*>(ws + P.off_phases);
    A.nphases = (int)P.phases.size();
    A.ctrl = reinterpret_cast<BatchCtrl*>(ws + P.off_ctrl);
    A.wavelet = reinterpret_cast<const float*>(ws + P.off_wav);
    A.ckpt_every = p->ckpt_every;
    A.image_every = p->image_every;
    A.nt = p->nt;
    A.timeout_cycles = (long long)((double)clock_khz * 1000.0 * g_wait_seconds);
    A.status = reinterpret_cast<int*>(ws);
    A.poison_shot = g_poison_shot;

    // capture on a private stream (the caller's may be the legacy default
    // stream, which cannot be captured); the graph runs on the caller's stream
    cudaStream_t cs = nullptr;
    CUB(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    {
        cudaError_t eb = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (eb != cudaSuccess) {
            cudaStreamDestroy(cs);
            return (rtm_status)set_error(RTM_ERR_CUDA, "batch capture: %s", cudaGetErrorString(eb));
        }
    }
    const cudaStream_t s_caller = s;
    s = cs;
    cudaError_t err = cudaSuccess;
    for (size_t wi = 0; wi < P.waves.size(); wi++) {
        const auto& w = P.waves[wi];
        A.zchunk = wave_zc[wi];
        long long items = 0;
        for (int i = w.first; i < w.second && err == cudaSuccess; i++) {
            const BatchShot& b = P.shots[i];
            items += b.ntiles;
            err = launch_batch_prep(b, d_vel, p->nx, p->ny, h_shots[i].ox, h_shots[i].oy,
                                    h_shots[i].oz, p->dt, const_cast<float*>(b.c),
                                    const_cast<float*>(b.gx), const_cast<float*>(b.gy),
                                    const_cast<float*>(b.gz), s);
            if (err == cudaSuccess)
                err = cudaMemsetAsync(b.img, 0, 4 * (size_t)b.nz * b.ny * b.NX, s);
        }
        if (err != cudaSuccess) break;
        err = cudaMemsetAsync(A.ctrl, 0, sizeof(BatchCtrl), s);
        if (err != cudaSuccess) break;
        A.shots = reinterpret_cast<const BatchShot*>(ws + P.off_desc) + w.first;
        A.nshots = w.second - w.first;
        A.items_per_phase = items;
        if (tma) {
            // the launch arguments carry each shot's tensor maps
            T->a = A;
            const int nseg = (p->nt + p->ckpt_every - 1) / p->ckpt_every;
            const int nfields = 5 + 2 * (nseg > 1 ? nseg - 1 : 0);
            for (int i = w.first; i < w.second && err == cudaSuccess; i++)
                err = batch_tma_maps(p->radius, rows, P.shots[i], nfields, p->ckpt_every + 1,
                                     T->maps[i - w.first]);
            if (err == cudaSuccess) err = launch_batch_tma(p->radius, rows, *T, nsm * bps, s);
        } else {
            err = launch_batch(p->radius, A, nsm * bps, s);
        }
        for (int i = w.first; i < w.second && err == cudaSuccess; i++)
            err = launch_batch_image_add(P.shots[i], p->nx, p->ny, h_shots[i].ox, h_shots[i].oy,
                                         h_shots[i].oz, d_image, s);
        if (err != cudaSuccess) break;
    }
    cudaError_t ec = cudaStreamEndCapture(cs, &graph);
    cudaStreamDestroy(cs);
    s = s_caller;
    if (err != cudaSuccess || ec != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return (rtm_status)set_error(RTM_ERR_CUDA, "batch graph capture failed: %s",
                                     cudaGetErrorString(err != cudaSuccess ? err : ec));
    }
    cudaGraphExec_t exec = nullptr;
    cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess)
        return (rtm_status)set_error(RTM_ERR_CUDA, "batch graph instantiate failed: %s",
                                     cudaGetErrorString(ei));
    cudaError_t el = cudaGraphLaunch(exec, s);
    cudaError_t es = el == cudaSuccess ? cudaStreamSynchronize(s) : el;
    cudaGraphExecDestroy(exec);
    if (es != cudaSuccess)
        return (rtm_status)set_error(RTM_ERR_CUDA, "batch graph failed: %s", cudaGetErrorString(es));
    int h_status = 0;
    CUB(cudaMemcpy(&h_status, ws, sizeof(int), cudaMemcpyDeviceToHost));
    if (h_status == RTM_ERR_TIMEOUT)
        return (rtm_status)set_error(RTM_ERR_TIMEOUT,
                                     "a persistent-kernel wait ran out after %.3g s; the batch "
                                     "was abandoned", g_wait_seconds);
    return RTM_OK;
}

}  // extern "C"
