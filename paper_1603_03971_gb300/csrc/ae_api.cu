// C ABI of the snapshot-compression autoencoder: encode, decode, one training
// step (forward, loss, hand-written backward, Adam) and the tensor-core GEMM
// engine self-check.

#include <stdint.h>
#include <string.h>

#include "../../include/rtm.h"
#include "ae_internal.h"
#include "rtm_internal.h"

using namespace rtm;
using namespace rtm::ae;

namespace {

constexpr size_t kAl = 256;
constexpr float kGradClip = 1.0f;  // global gradient-norm bound of each Adam step
size_t upa(size_t v) { return (v + kAl - 1) / kAl * kAl; }

struct AeLayout {
    size_t status = 0, scalars = 64;
    size_t h1, lat, g1, y, gy, ga3, glat, ga1, grad, total;
};

AeLayout ae_layout(int nx, int ny, int nz) {
    const size_t n = (size_t)nx * ny * nz, nh = n / 8, nl = n / 64;
    AeLayout L;
    size_t o = kAl;
    auto take = [&](size_t b) {
        size_t r = o;
        o += upa(b);
        return r;
    };
    L.h1 = take(nh * 32 * 2);
    L.lat = take(nl * 16 * 2);
    L.g1 = take(nh * 32 * 2);
    L.y = take(n * 4);
    L.gy = take(n * 2);
    L.ga3 = take(nh * 32 * 2);
    L.glat = take(nl * 16 * 2);
    L.ga1 = take(nh * 32 * 2);
    L.grad = take((size_t)kNParams * 4);
    L.total = o;
    return L;
}

rtm_status check_dims(int nx, int ny, int nz) {
    if (nx < 4 || ny < 4 || nz < 4 || nx % 4 || ny % 4 || nz % 4)
        return (rtm_status)set_error(RTM_ERR_INVALID,
                                     "codec volume %dx%dx%d: every side must be a positive "
                                     "multiple of 4",
                                     nx, ny, nz);
    if ((long long)nx * ny * nz > (1LL << 34))
        return (rtm_status)set_error(RTM_ERR_INVALID, "codec volume too large");
    return RTM_OK;
}

rtm_status check_ws(void* ws, size_t bytes, size_t need) {
    if (!ws || ((uintptr_t)ws % kAl))
        return (rtm_status)set_error(RTM_ERR_WORKSPACE, "codec workspace NULL or not 256-byte aligned");
    if (bytes < need)
        return (rtm_status)set_error(RTM_ERR_WORKSPACE, "codec workspace %zu bytes, %zu needed", bytes,
                                     need);
    return RTM_OK;
}

#define CUA(call)                                                                              \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return (rtm_status)set_error(RTM_ERR_CUDA, "%s failed: %s", #call,                 \
                                         cudaGetErrorString(e_));                              \
    } while (0)

}  // namespace

extern "C" {

size_t rtm_ae_param_count(void) { return (size_t)kNParams; }

size_t rtm_ae_workspace_size(int32_t nx, int32_t ny, int32_t nz) {
    if (check_dims(nx, ny, nz) != RTM_OK) return 0;
    return ae_layout(nx, ny, nz).total;
}

rtm_status rtm_ae_encode(const float* d_params, const float* d_snap, int64_t sy, int64_t sz,
                         int32_t nx, int32_t ny, int32_t nz, uint16_t* d_latent, float* d_scale,
                         void* d_ws, size_t ws_bytes, rtm_stream stream) {
    rtm_status st = check_dims(nx, ny, nz);
    if (st != RTM_OK) return st;
    const AeLayout L = ae_layout(nx, ny, nz);
    if ((st = check_ws(d_ws, ws_bytes, L.total)) != RTM_OK) return st;
    if (!d_params || !d_snap || !d_latent || ((uintptr_t)d_latent % 16))
        return (rtm_status)set_error(RTM_ERR_INVALID, "codec arrays NULL or latent not 16-byte aligned");
    if (sy < nx || sz < sy * ny)
        return (rtm_status)set_error(RTM_ERR_INVALID, "snapshot strides overlap rows or planes");
    char* w = reinterpret_cast<char*>(d_ws);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaGetLastError();
    const Vol in{const_cast<float*>(d_snap), sy, sz, nx, ny, nz};
    CUA(cudaMemsetAsync(w, 0, sizeof(int), s));
    CUA(ae_encode(d_params, in, reinterpret_cast<bf16*>(w + L.h1), reinterpret_cast<bf16*>(d_latent),
                  reinterpret_cast<AeScalars*>(w + L.scalars), d_scale,
                  reinterpret_cast<int*>(w + L.status), s));
    return RTM_OK;
}

rtm_status rtm_ae_decode(const float* d_params, const uint16_t* d_latent, const float* d_scale,
                         float* d_out, int64_t sy, int64_t sz, int32_t nx, int32_t ny, int32_t nz,
                         void* d_ws, size_t ws_bytes, rtm_stream stream) {
    rtm_status st = check_dims(nx, ny, nz);
    if (st != RTM_OK) return st;
    const AeLayout L = ae_layout(nx, ny, nz);
    if ((st = check_ws(d_ws, ws_bytes, L.total)) != RTM_OK) return st;
    if (!d_params || !d_latent || !d_out || ((uintptr_t)d_latent % 16))
        return (rtm_status)set_error(RTM_ERR_INVALID, "codec arrays NULL or latent not 16-byte aligned");
    if (sy < nx || sz < sy * ny)
        return (rtm_status)set_error(RTM_ERR_INVALID, "output strides overlap rows or planes");
    char* w = reinterpret_cast<char*>(d_ws);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaGetLastError();
    const Vol out{d_out, sy, sz, nx, ny, nz};
    CUA(cudaMemsetAsync(w, 0, sizeof(int), s));
    CUA(ae_decode(d_params, reinterpret_cast<const bf16*>(d_latent), d_scale, out, nullptr,
                  reinterpret_cast<int*>(w + L.status), s));
    return RTM_OK;
}

rtm_status rtm_ae_train_step(float* d_params, float* d_adam_m, float* d_adam_v, int32_t step,
                             float lr, const float* d_batch, int32_t batch, int32_t nx,
                             int32_t ny, int32_t nz, double* d_loss, float* d_grad, void* d_ws,
                             size_t ws_bytes, rtm_stream stream) {
    rtm_status st = check_dims(nx, ny, nz);
    if (st != RTM_OK) return st;
    const AeLayout L = ae_layout(nx, ny, nz);
    if ((st = check_ws(d_ws, ws_bytes, L.total)) != RTM_OK) return st;
    if (!d_params || !d_batch || batch < 1 || !d_loss)
        return (rtm_status)set_error(RTM_ERR_INVALID, "training arrays NULL or batch < 1");
    if (lr > 0.f && (!d_adam_m || !d_adam_v || step < 1))
        return (rtm_status)set_error(RTM_ERR_INVALID, "Adam needs moment buffers and step >= 1");
    char* w = reinterpret_cast<char*>(d_ws);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaGetLastError();
    float* grad = reinterpret_cast<float*>(w + L.grad);
    AeTrainBufs b{reinterpret_cast<bf16*>(w + L.h1),  reinterpret_cast<bf16*>(w + L.lat),
                  reinterpret_cast<bf16*>(w + L.g1),  reinterpret_cast<bf16*>(w + L.gy),
                  reinterpret_cast<bf16*>(w + L.ga3), reinterpret_cast<bf16*>(w + L.glat),
                  reinterpret_cast<bf16*>(w + L.ga1), reinterpret_cast<float*>(w + L.y)};
    CUA(cudaMemsetAsync(w, 0, sizeof(int), s));
    CUA(cudaMemsetAsync(grad, 0, sizeof(float) * kNParams, s));
    CUA(cudaMemsetAsync(d_loss, 0, sizeof(double), s));
    const size_t n = (size_t)nx * ny * nz;
    for (int i = 0; i < batch; i++) {
        const Vol in{const_cast<float*>(d_batch) + i * n, (long long)nx, (long long)nx * ny, nx,
                     ny, nz};
        CUA(ae_sample_grad(d_params, in, 1.0f / (float)batch, b,
                           reinterpret_cast<AeScalars*>(w + L.scalars), d_loss, grad,
                           reinterpret_cast<int*>(w + L.status), s));
    }
    if (d_grad)
        CUA(cudaMemcpyAsync(d_grad, grad, sizeof(float) * kNParams, cudaMemcpyDeviceToDevice, s));
    if (lr > 0.f)
        CUA(ae_adam(d_params, d_adam_m, d_adam_v, grad, step, lr, kGradClip,
                    reinterpret_cast<double*>(w + L.scalars + 128), s));
    return RTM_OK;
}

rtm_status rtm_ae_gemm_bf16(const uint16_t* d_A, const uint16_t* d_B, float* d_C, int32_t M,
                            int32_t K, int32_t N, int32_t* d_status, rtm_stream stream) {
    if (!d_A || !d_B || !d_C || M < 1 || K < 32 || K % 32 || (N != 16 && N != 32))
        return (rtm_status)set_error(RTM_ERR_INVALID, "gemm: M >= 1, K a multiple of 32, N 16 or 32");
    if (((uintptr_t)d_A % 16) || ((uintptr_t)d_B % 16))
        return (rtm_status)set_error(RTM_ERR_INVALID, "gemm operands not 16-byte aligned");
    GemmArgs a{reinterpret_cast<const bf16*>(d_A), reinterpret_cast<const bf16*>(d_B), d_C, M, K};
    CUA(ae_gemm_test(a, N, reinterpret_cast<int*>(d_status), reinterpret_cast<cudaStream_t>(stream)));
    return RTM_OK;
}

rtm_status rtm_ae_set_encoder(int32_t which) {
    if (which < 0 || which > 2)
        return (rtm_status)set_error(RTM_ERR_INVALID, "encoder: 0 automatic, 1 GEMM engine, 2 z-marching");
    ae_set_encoder(which);
    return RTM_OK;
}

rtm_status rtm_ae_set_decoder(int32_t which) {
    if (which < 0 || which > 2)
        return (rtm_status)set_error(RTM_ERR_INVALID, "decoder: 0 automatic, 1 GEMM engine, 2 z-marching");
    ae_set_decoder(which);
    return RTM_OK;
}

}  // extern "C"
