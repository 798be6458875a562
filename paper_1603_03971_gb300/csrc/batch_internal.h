// Internal declarations of the batched multi-shot RTM kernel.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rtm_internal.h"

namespace rtm {

constexpr int kMaxBatchShots = 64;

// one shot of a wave: its padded aperture grid and its buffers
struct BatchShot {
    int NX, NY, NZ, nb, nx, ny, nz;
    int tiles_x, tiles_y, tiles_z, ntiles;
    int src_x, src_y, src_z;  // padded coordinates
    int rec_z;                // padded z of the receiver plane (every model x, y)
    long long item_base;      // first tile of this shot within one phase step
    // padded fields, fstride floats apart: c, f0, f1, m0, m1, then the
    // (nseg - 1) checkpoints of two fields (field 5 + 2 (j - 1) + w)
    long long fstride;
    const float* c;
    float *f0, *f1, *m0, *m1;  // forward and backward field pairs
    float* ckpt;               // checkpoint j, field w: ckpt + (2 (j - 1) + w) fstride
    // slabs [nz][ny][NX], sstride floats apart: ckpt_every snapshots, then the image
    long long sstride;
    float* snap;
    float* img;                // snap + ckpt_every sstride
    const float *gx, *gy, *gz;
    const float* dobs;         // [nt][ny][nx] data injected backward
    float* data;               // [nt][ny][nx] modelled data, or NULL
};

// phase step of the common schedule: forward steps, then per checkpoint
// segment (last first) its recompute steps and its backward steps
enum BatchPhaseKind { PH_FWD = 0, PH_REC = 1, PH_BWD = 2 };
struct BatchPhase {
    int kind;
    int step;   // n (forward, recompute) or m (backward)
    int seg;    // checkpoint segment j (recompute, backward)
    int local;  // n - n0 (recompute) or m - 1 - n0 (backward): the snapshot slot
};

struct BatchCtrl {
    unsigned long long next;  // work-queue head
    int abort;                // set when a bounded wait ran out
    int status;               // RTM_ERR_TIMEOUT if so
    unsigned int done[kMaxBatchShots];  // completed tiles per shot
};

struct BatchArgs {
    const BatchShot* shots;
    int nshots;
    const BatchPhase* phases;
    int nphases;
    long long items_per_phase;
    BatchCtrl* ctrl;
    const float* wavelet;
    float a[kMaxRadius + 1];
    float inv_dx3;
    int zchunk, ckpt_every, image_every, nt;
    long long timeout_cycles;
    int* status;  // workspace status word (RTM_ERR_TIMEOUT on a wait that ran out)
    int poison_shot;  // >= 0: that shot's first item waits for a count nothing reaches
};

cudaError_t launch_batch(int radius, const BatchArgs& a, int grid, cudaStream_t s);

// the TMA form (batch_tma.cu): the launch arguments plus three tensor maps
// per shot of the wave (halo tile and plain tile over the field stack, plain
// tile over the slab stack)
struct BatchTmaArgs {
    BatchArgs a;
    CUtensorMap maps[kMaxBatchShots][3];
};
// tile_rows: 16 (256-thread blocks) or 8 (128-thread blocks)
int batch_tma_tile_x(int radius, int tile_rows);
int batch_tma_blocks_per_sm(int radius, int tile_rows);
cudaError_t batch_tma_maps(int radius, int tile_rows, const BatchShot& b, int nfields,
                           int nslabs, CUtensorMap* maps);
cudaError_t launch_batch_tma(int radius, int tile_rows, const BatchTmaArgs& a, int grid,
                             cudaStream_t s);
int batch_blocks_per_sm(int radius);
cudaError_t launch_batch_prep(const BatchShot& sh, const float* vel_full, int full_nx, int full_ny,
                              int ox, int oy, int oz, double dt, float* c, float* gx, float* gy,
                              float* gz, cudaStream_t s);
cudaError_t launch_batch_image_add(const BatchShot& sh, int full_nx, int full_ny, int ox, int oy,
                                   int oz, float* image_full, cudaStream_t s);

}  // namespace rtm
