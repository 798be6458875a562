// Internal declarations of the snapshot-compression autoencoder.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace rtm {
namespace ae {

// offsets of the parameters in the flat float32 vector
constexpr int kOW1 = 0;       // W1[32][2][2][2]
constexpr int kOB1 = 256;     // b1[32]
constexpr int kOW2 = 288;     // W2[16][3][3][3][32]
constexpr int kOB2 = 14112;   // b2[16]
constexpr int kOW3 = 14128;   // W3[32][4][4][4][16]
constexpr int kOB3 = 46896;   // b3[32]
constexpr int kOW4 = 46928;   // W4[2][2][2][32]
constexpr int kOB4 = 47184;   // b4[1]
constexpr int kNParams = 47185;
constexpr float kSlope = 0.1f;  // LeakyReLU

struct Dims3 {
    int nx, ny, nz;
};

// strided float32 volume, x contiguous
struct Vol {
    float* p;
    long long sy, sz;
    int nx, ny, nz;
};

using bf16 = __nv_bfloat16;

struct GemmArgs { const bf16* A; const bf16* B; float* C; int M, K; };
struct E1Args { Vol in; const float* inv_sigma; const float* P; bf16* h1; Dims3 h; };
struct E2Args { const bf16* h1; Dims3 h; const float* P; bf16* lat; Dims3 l; };
struct D1Args { const bf16* lat; Dims3 l; const float* P; bf16* g1; Dims3 h; };
struct D2Args { const bf16* g1; Dims3 h; const float* P; const float* sigma; Vol out; };
struct D12Args { D1Args d1; const float* sigma; Vol out; };
struct D2dArgs { const bf16* gy; Dims3 h; const bf16* g1; const float* P; bf16* ga3; };
struct D1dArgs { const bf16* ga3; Dims3 h; Dims3 l; const float* P; bf16* glat; };
struct E2dArgs { const bf16* glat; Dims3 l; const bf16* h1; Dims3 h; const float* P; bf16* ga1; };
struct E2wArgs { const bf16* h1; Dims3 h; const bf16* glat; Dims3 l; float* grad; int chunks_per_cta; };
struct D1wArgs { const bf16* lat; Dims3 l; const bf16* ga3; Dims3 h; float* grad; int chunks_per_cta; };

// device-resident scalars of one codec call
struct AeScalars {
    double sumsq;
    float sigma;
    float inv_sigma;
    double loss;
};

struct AeTrainBufs {
    bf16 *h1, *lat, *g1, *gy, *ga3, *glat, *ga1;
    float* y;
};

}  // namespace ae

cudaError_t ae_gemm_test(const ae::GemmArgs& a, int N, int* status, cudaStream_t s);
cudaError_t ae_rms(const ae::Vol& in, ae::AeScalars* sc, cudaStream_t s);
// snapshot -> latent; the snapshot's rms goes to sigma_out if given. With
// keep_h1 the GEMM-engine layers run and leave E1's output in h1 (training
// reads it); otherwise the z-marching kernel runs where it can and h1 is
// untouched scratch. With sumsq_ready, sc->sumsq already holds the
// snapshot's sum of squares (accumulated by the stencil step that wrote it)
// and only the scale is derived from it.
cudaError_t ae_encode(const float* P, const ae::Vol& in, ae::bf16* h1, ae::bf16* lat,
                      ae::AeScalars* sc, float* sigma_out, int* status, cudaStream_t s,
                      bool keep_h1 = false, bool sumsq_ready = false);
// latent -> snapshot scaled by *sigma (1 if NULL); with g1 NULL the two
// decoder layers run fused (inference), otherwise g1 keeps the D1 output
cudaError_t ae_decode(const float* P, const ae::bf16* lat, const float* sigma, const ae::Vol& out,
                      ae::bf16* g1, int* status, cudaStream_t s);
// the fused inference decoder as one z-marching persistent kernel (TMA plane
// loads read in place by the tensor cores); cudaErrorNotSupported when it
// cannot run or is not selected
cudaError_t ae_decode_march(const ae::D12Args& a, int* status, cudaStream_t s);
// 0 automatic, 1 GEMM-engine decoder, 2 z-marching decoder
void ae_set_decoder(int which);
// E1 + E2 as one z-marching persistent kernel (h1 kept in shared memory);
// cudaErrorNotSupported when it cannot run or is not selected
cudaError_t ae_encode_march(const float* P, const ae::Vol& in, const float* inv_sigma,
                            ae::bf16* lat, int* status, cudaStream_t s);
// 0 automatic, 1 GEMM-engine encoder, 2 z-marching encoder
void ae_set_encoder(int which);
cudaError_t ae_sample_grad(const float* P, const ae::Vol& in, float scale,
                           const ae::AeTrainBufs& b, ae::AeScalars* sc, double* loss, float* grad,
                           int* status, cudaStream_t s);
// Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) with the gradient
// scaled down to a global L2 norm of clip when it is larger (clip <= 0: off)
cudaError_t ae_adam(float* P, float* m, float* v, const float* g, int step, float lr, float clip,
                    double* scratch, cudaStream_t s);

}  // namespace rtm
