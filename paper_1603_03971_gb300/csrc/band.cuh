// Boundary band of the model region, for source-wavefield reconstruction by
// reverse time stepping.
//
// Inside the model region the sponge factor is exactly 1, so the forward
// update u^{n+1} = (2 u^n + c L u^n) - u^{n-1} can be solved for u^{n-1}:
// the same arithmetic with the two time levels swapped. A cell whose whole
// star lies in the model region (at least r cells from every face) is
// recovered that way; the cells within r of a face (the band) need stencil
// neighbours in the sponge, whose state cannot be run backwards, so the
// forward pass stores the band of every state and the reverse pass reads it.
//
// Band storage per state, model coordinates, nx, ny, nz > 2r:
//   2r z-face planes           [2r][ny][nx]           mz < r or mz >= nz - r
//   2r y-face rows per plane   [nz - 2r][2r][nx]      other planes, my < r or my >= ny - r
//   2r x-face cells per row    [nz - 2r][ny - 2r][2r] the rest, mx < r or mx >= nx - r
#pragma once

#include <cuda_runtime.h>

namespace rtm {

__host__ __device__ inline long long band_cells(int nx, int ny, int nz, int r) {
    const long long r2 = 2LL * r;
    return r2 * nx * ny + r2 * (nz - r2) * nx + r2 * (nz - r2) * (ny - r2);
}

// offset of model cell (mx, my, mz) in one state's band, -1 for an inner
// cell; the caller keeps the cell inside the model region
__host__ __device__ inline long long band_offset(int mx, int my, int mz, int nx, int ny, int nz,
                                                 int r) {
    const int fz = mz < r ? mz : (mz >= nz - r ? mz - (nz - 2 * r) : -1);
    if (fz >= 0) return ((long long)fz * ny + my) * nx + mx;
    const long long zi = mz - r;
    long long base = 2LL * r * ny * nx;
    const int fy = my < r ? my : (my >= ny - r ? my - (ny - 2 * r) : -1);
    if (fy >= 0) return base + (zi * 2 * r + fy) * nx + mx;
    base += (long long)(nz - 2 * r) * 2 * r * nx;
    const int fx = mx < r ? mx : (mx >= nx - r ? mx - (nx - 2 * r) : -1);
    if (fx >= 0) return base + (zi * (ny - 2 * r) + (my - r)) * 2 * r + fx;
    return -1;
}

// model cell of band offset b, 0 <= b < band_cells (the inverse of band_offset)
__host__ __device__ inline void band_cell(long long b, int nx, int ny, int nz, int r, int& mx,
                                          int& my, int& mz) {
    const long long r2 = 2LL * r;
    const long long zface = r2 * ny * nx;
    if (b < zface) {
        const long long fz = b / ((long long)ny * nx), rem = b - fz * ny * nx;
        mz = (int)(fz < r ? fz : fz + nz - r2);
        my = (int)(rem / nx);
        mx = (int)(rem - (long long)my * nx);
        return;
    }
    b -= zface;
    const long long yface = (nz - r2) * r2 * nx;
    if (b < yface) {
        const long long zi = b / (r2 * nx), rem = b - zi * r2 * nx;
        const int fy = (int)(rem / nx);
        mz = (int)(zi + r);
        my = fy < r ? fy : fy + ny - (int)r2;
        mx = (int)(rem - (long long)fy * nx);
        return;
    }
    b -= yface;
    const long long row = (ny - r2) * r2;
    const long long zi = b / row, rem = b - zi * row;
    const int yi = (int)(rem / r2), fx = (int)(rem - yi * r2);
    mz = (int)(zi + r);
    my = yi + r;
    mx = fx < r ? fx : fx + nx - (int)r2;
}

}  // namespace rtm
