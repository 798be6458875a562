// rtm_forward_noalloc: forward modelling whose scratch lives in a fixed
// static device array instead of a caller-provided workspace.
//
// For callers that cannot allocate device memory: code running inside a
// host framework that owns every allocation, plugins loaded into a process
// whose allocator they may not touch, or tools that must not change the
// device's memory footprint while they run. They pass only the inputs and
// outputs; the two wavefields, the wavelet, the sponge profiles and the status
// word live in kNoAllocBytes of file-scope device memory that every GPU which
// loads this library holds until the process exits.

#include <math.h>
#include <string.h>

#include <mutex>

#include "../../include/rtm.h"
#include "rtm_internal.h"

using namespace rtm;

namespace {

constexpr size_t kNoAllocBytes = RTM_NOALLOC_SCRATCH_BYTES;
constexpr size_t kAlignNA = 256;
constexpr int kMaxDevices = 64;

// The scratch itself. Host code may only use its address as returned by
// cudaGetSymbolAddress on the current device; the name alone is a host-side
// stand-in, not a device address.
static __device__ __align__(256) unsigned char g_scratch[kNoAllocBytes];

std::mutex g_na_mu;
void* g_na_ptr[kMaxDevices] = {nullptr};

size_t up_na(size_t v) { return (v + kAlignNA - 1) / kAlignNA * kAlignNA; }

// a failed CUDA call returns RTM_ERR_CUDA with its message in rtm_last_error()
#define NA_CU(call)                                                                    \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return (rtm_status)set_error(RTM_ERR_CUDA, "rtm_forward_noalloc: %s failed: %s", \
                                         #call, cudaGetErrorString(e_));               \
    } while (0)

// The scratch's device address on the current device, looked up once per device.
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_na_ptr[dev] = p;
    }
    *out = g_na_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" rtm_status rtm_forward_noalloc(const rtm_params* p, const float* d_c,
                                          const int32_t* d_rec, float* d_data,
                                          float* d_u_last, rtm_stream stream) {
    rtm_status st = rtm_validate(p);
    if (st != RTM_OK) return st;
    if (!d_c || ((uintptr_t)d_c % 16))
        return (rtm_status)set_error(RTM_ERR_INVALID, "coefficient grid NULL or not 16-byte aligned");
    if (p->nrec > 0 && !d_rec)
        return (rtm_status)set_error(RTM_ERR_INVALID, "receiver array is NULL");
    if (d_u_last && ((uintptr_t)d_u_last % 16))
        return (rtm_status)set_error(RTM_ERR_INVALID, "u_last not 16-byte aligned");

    const int NX = p->nx + 2 * p->nb, NY = p->ny + 2 * p->nb, NZ = p->nz + 2 * p->nb;
    const size_t N = (size_t)NX * NY * NZ;
    // scratch layout: status block, wavelet, three sponge profiles, two fields
    const size_t o_status = 0;
    const size_t o_wav = o_status + kAlignNA;
    const size_t o_gx = o_wav + up_na(sizeof(float) * (size_t)p->nt);
    const size_t o_gy = o_gx + up_na(sizeof(float) * NX);
    const size_t o_gz = o_gy + up_na(sizeof(float) * NY);
    const size_t o_f0 = o_gz + up_na(sizeof(float) * NZ);
    const size_t o_f1 = o_f0 + up_na(sizeof(float) * N);
    const size_t need = o_f1 + up_na(sizeof(float) * N);
    if (need > kNoAllocBytes)
        return (rtm_status)set_error(
            RTM_ERR_WORKSPACE,
            "rtm_forward_noalloc: %zu bytes of scratch needed (two %dx%dx%d fields), the static "
            "scratch holds %zu; use rtm_forward with a workspace",
            need, NX, NY, NZ, (size_t)kNoAllocBytes);

    cudaGetLastError();  // a stale error of the caller's earlier work is not ours
    void* base = nullptr;
    cudaError_t ea = scratch_address(&base);
    if (ea != cudaSuccess)
        return (rtm_status)set_error(RTM_ERR_CUDA, "cudaGetSymbolAddress of the scratch failed: %s",
                                     cudaGetErrorString(ea));
    char* s8 = reinterpret_cast<char*>(base);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int* status = reinterpret_cast<int*>(s8 + o_status);
    float* wav = reinterpret_cast<float*>(s8 + o_wav);
    float* gx = reinterpret_cast<float*>(s8 + o_gx);
    float* gy = reinterpret_cast<float*>(s8 + o_gy);
    float* gz = reinterpret_cast<float*>(s8 + o_gz);
    float* prev = reinterpret_cast<float*>(s8 + o_f0);
    float* cur = reinterpret_cast<float*>(s8 + o_f1);

    // the array keeps the previous call's contents: clear what starts at zero
    NA_CU(cudaMemsetAsync(status, 0, sizeof(int), s));
    NA_CU(cudaMemsetAsync(prev, 0, sizeof(float) * N, s));
    NA_CU(cudaMemsetAsync(cur, 0, sizeof(float) * N, s));

    Geometry G{NX, NY, NZ, p->nb, p->nx, p->ny, p->nz};
    NA_CU(launch_wavelet(p->nt, p->dt, p->f0, p->t0, wav, s));
    NA_CU(launch_sponge(G, gx, gy, gz, s));

    StepArgs A;
    memset(&A, 0, sizeof A);
    step_weights(p->radius, p->dx, A.a);
    A.c = d_c;
    A.gx = gx;
    A.gy = gy;
    A.gz = gz;
    A.NX = NX;
    A.NY = NY;
    A.NZ = NZ;
    A.nb = p->nb;
    A.nx = p->nx;
    A.ny = p->ny;
    A.nz = p->nz;
    // the slab height set by rtm_set_tuning applies; the plane loads are
    // always the vector-load kernel's
    const int zc = tuning_zchunk(p->radius, MODE_FWD);
    A.zchunk = zc > 0 ? zc : auto_zchunk(p->radius, NX, NY, NZ);
    if ((NZ + A.zchunk - 1) / A.zchunk > 65535) A.zchunk = (NZ + 65534) / 65535;
    set_region(A, MODE_FWD);

    const long long src = ((long long)(p->src_z + p->nb) * NY + (p->src_y + p->nb)) * NX +
                          (p->src_x + p->nb);
    const float inv_dx3 = (float)(1.0 / (p->dx * p->dx * p->dx));
    for (int n = 0; n < p->nt; n++) {
        float* row = (d_data && n >= 1) ? d_data + (size_t)(n - 1) * p->nrec : nullptr;
        NA_CU(launch_fwd_aux(G, cur, prev, d_c, gx, gy, gz, d_rec, p->nrec, row, src, wav + n,
                             inv_dx3, status, s));
        A.u_cur = cur;
        A.u_prev = prev;
        NA_CU(launch_stencil(p->radius, MODE_FWD, A, s));
        float* t = prev;
        prev = cur;
        cur = t;
    }
    if (d_data)
        NA_CU(launch_fwd_aux(G, cur, prev, d_c, gx, gy, gz, d_rec, p->nrec,
                             d_data + (size_t)(p->nt - 1) * p->nrec, src, nullptr, inv_dx3,
                             status, s));
    if (d_u_last) {
        NA_CU(cudaMemcpyAsync(d_u_last, prev, sizeof(float) * N, cudaMemcpyDeviceToDevice, s));
        NA_CU(cudaMemcpyAsync(d_u_last + N, cur, sizeof(float) * N, cudaMemcpyDeviceToDevice, s));
    }
    return RTM_OK;
}
