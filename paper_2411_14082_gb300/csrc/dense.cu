// Dense tail of the re-factorization.
//
// When the last m columns of the factor form a structurally dense block
// (every column k >= p = n-m holds every row >= p), the column kernels apply
// to those columns only their dependencies before p and leave the rows >= p
// in S (m x m, column-major).  S is then the Schur complement of the block,
// and its factorization is a dense LU with the pivot sequence fixed (the
// block's rows are already in step order) and the same check per column as
// the sparse columns (Section IV-B, Algorithms 3 and 4):
//     fail iff x(k) == 0 or |x(k)| < eps * max |x(rows > k)|.
// It runs blocked right-looking, panels of kDenseNb columns:
//   panel  - one CTA loads the panel (rows c0..m-1) into shared memory and
//            factors it column by column (check, scale, rank-1 update of the
//            panel's later columns), then computes the panel's rows of U for
//            every trailing column (unit lower triangular solve with L11);
//   update - the trailing block S(c0+nb:m, c0+nb:m) -= L21 * U12, in 64 x 64
//            tiles, 4 x 4 per thread (FP64 fused multiply-adds).
// A failed check sets `interrupted` and `first_bad`; every later kernel then
// returns at once and the block's columns stay unfinished, so the restart
// recomputes them with pivoting (Section IV-C).  The scatter copies the
// block into the factor's columns and publishes their ready flags.
#include <cuda_runtime.h>

#include <cstdint>

#include "device_util.cuh"
#include "gblu_internal.h"

namespace gblu {

namespace {

using namespace dev;

constexpr int kNb = kDenseNb;
constexpr int kPanelThreads = 1024;
constexpr int kTile = 64;
constexpr int kTileThreads = 256;

__device__ __forceinline__ bool dense_stopped(const DevCtl *ctl)
{
    return ld_volatile(&ctl->interrupted) != 0 || ld_volatile(&ctl->status) != 0;
}

// factor panel [c0, c0+w) of S and compute U12 = L11^{-1} S(c0:c0+w, c0+w:m)
__global__ void __launch_bounds__(kPanelThreads) dense_panel_kernel(DenseArgs2 d, int c0)
{
    __shared__ double s_red[32];
    __shared__ int s_fail;
    if (dense_stopped(d.ctl)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    double *P = reinterpret_cast<double *>(smem);   // panel column c at P[c * R], rows c0 .. m-1
    const int R = d.m - c0, w = min(kNb, R);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int idx = tid; idx < w * R; idx += kPanelThreads) {
        const int c = idx / R, r = idx - c * R;
        P[idx] = d.S[(int64_t)(c0 + c) * d.ld + c0 + r];
    }
    if (tid == 0) s_fail = 0;
    __syncthreads();
    for (int c = 0; c < w; c++) {
        double *col = P + (size_t)c * R;
        double mx = 0.0;
        for (int r = c + 1 + tid; r < R; r += kPanelThreads) mx = max_nan(mx, fabs(col[r]));
        mx = warp_max(mx);
        if (lane == 0) s_red[wid] = mx;
        __syncthreads();
        if (wid == 0) {
            double v = s_red[lane];
            v = warp_max(v);
            if (lane == 0) {
                const double piv = col[c];
                if (!((piv != 0.0) && isfinite(piv) && (fabs(piv) >= d.eps * v))) {
                    s_fail = 1;
                    atomicExch(&d.ctl->interrupted, 1);
                    atomicMin(&d.ctl->first_bad, d.p + c0 + c);
                }
            }
        }
        __syncthreads();
        if (s_fail) return;
        const double inv = 1.0 / col[c];
        for (int r = c + 1 + tid; r < R; r += kPanelThreads) col[r] *= inv;
        __syncthreads();
        const int nc = w - c - 1, nr = R - c - 1;   // rank-1 update of the panel's later columns
        for (int idx = tid; idx < nc * nr; idx += kPanelThreads) {
            const int cc = c + 1 + idx / nr, r = c + 1 + idx % nr;
            double *pc = P + (size_t)cc * R;
            pc[r] = fma(-col[r], pc[c], pc[r]);
        }
        __syncthreads();
    }
    for (int idx = tid; idx < w * R; idx += kPanelThreads) {
        const int c = idx / R, r = idx - c * R;
        d.S[(int64_t)(c0 + c) * d.ld + c0 + r] = P[idx];
    }
    // U12: rows c0 .. c0+w-1 of every trailing column, forward substitution
    for (int j = c0 + w + tid; j < d.m; j += kPanelThreads) {
        double *sj = d.S + (int64_t)j * d.ld + c0;
        double u[kNb];
#pragma unroll
        for (int i = 0; i < kNb; i++) u[i] = i < w ? sj[i] : 0.0;
#pragma unroll
        for (int i = 1; i < kNb; i++) {
#pragma unroll
            for (int c = 0; c < kNb - 1; c++)
                if (c < i && i < w) u[i] = fma(-P[(size_t)c * R + i], u[c], u[i]);
        }
#pragma unroll
        for (int i = 0; i < kNb; i++)
            if (i < w) sj[i] = u[i];
    }
}

// S(t0:m, t0:m) -= S(t0:m, c0:t0) * S(c0:t0, t0:m), t0 = c0 + kNb
__global__ void __launch_bounds__(kTileThreads) dense_update_kernel(DenseArgs2 d, int c0)
{
    __shared__ double Ls[kNb][kTile];   // L(rb + i, c0 + c)
    __shared__ double Us[kNb][kTile];   // U(c0 + c, cb + j)
    if (dense_stopped(d.ctl)) return;
    const int t0 = c0 + kNb;
    const int rb = t0 + blockIdx.y * kTile, cb = t0 + blockIdx.x * kTile;
    const int tid = threadIdx.x;
    for (int idx = tid; idx < kNb * kTile; idx += kTileThreads) {
        const int c = idx / kTile, i = idx % kTile;
        Ls[c][i] = rb + i < d.m ? d.S[(int64_t)(c0 + c) * d.ld + rb + i] : 0.0;
        const int j = idx / kNb, cu = idx % kNb;
        Us[cu][j] = cb + j < d.m ? d.S[(int64_t)(cb + j) * d.ld + c0 + cu] : 0.0;
    }
    __syncthreads();
    const int tx = tid & 15, ty = tid >> 4;   // rows tx + 16 a, columns ty + 16 b
    double acc[4][4];
#pragma unroll
    for (int b = 0; b < 4; b++) {
        const int j = cb + ty + 16 * b;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int r = rb + tx + 16 * q;
            acc[q][b] = (r < d.m && j < d.m) ? d.S[(int64_t)j * d.ld + r] : 0.0;
        }
    }
#pragma unroll
    for (int c = 0; c < kNb; c++) {
        double lv[4], uv[4];
#pragma unroll
        for (int q = 0; q < 4; q++) lv[q] = Ls[c][tx + 16 * q];
#pragma unroll
        for (int b = 0; b < 4; b++) uv[b] = Us[c][ty + 16 * b];
#pragma unroll
        for (int q = 0; q < 4; q++)
#pragma unroll
            for (int b = 0; b < 4; b++) acc[q][b] = fma(-lv[q], uv[b], acc[q][b]);
    }
#pragma unroll
    for (int b = 0; b < 4; b++) {
        const int j = cb + ty + 16 * b;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int r = rb + tx + 16 * q;
            if (r < d.m && j < d.m) d.S[(int64_t)j * d.ld + r] = acc[q][b];
        }
    }
}

// block column c -> factor column p + c (rows p .. n-1 start at slot s0[c]);
// then its ready flag
__global__ void __launch_bounds__(256) dense_scatter_kernel(DenseArgs2 d)
{
    if (dense_stopped(d.ctl)) return;
    const int c = blockIdx.x;
    const int64_t base = __ldg(d.LUp + d.p + c) + __ldg(d.s0 + c);
    const double *sc = d.S + (int64_t)c * d.ld;
    for (int r = threadIdx.x; r < d.m; r += blockDim.x) d.LUx[base + r] = sc[r];
    // the stores are ordered before the release by the barrier
    __syncthreads();
    if (threadIdx.x == 0) st_release(d.finish + d.p + c, d.epoch < 0 ? ld_volatile(&d.ctl->epoch) : d.epoch);
}

size_t panel_smem(int rows) { return (size_t)rows * kNb * sizeof(double); }

}  // namespace

int dense_setup(int max_rows)
{
    return (int)cudaFuncSetAttribute(dense_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)panel_smem(max_rows));
}

int launch_dense_lu(const DenseArgs2 &d, void *stream, long long *launches)
{
    cudaStream_t st = (cudaStream_t)stream;
    long long nl = 0;
    for (int c0 = 0; c0 < d.m; c0 += kNb) {
        dense_panel_kernel<<<1, kPanelThreads, panel_smem(d.m - c0), st>>>(d, c0);
        nl++;
        const int t0 = c0 + kNb;
        if (t0 < d.m) {
            const int nt = (d.m - t0 + kTile - 1) / kTile;
            dense_update_kernel<<<dim3(nt, nt), kTileThreads, 0, st>>>(d, c0);
            nl++;
        }
    }
    dense_scatter_kernel<<<d.m, 256, 0, st>>>(d);
    nl++;
    *launches = nl;
    return (int)cudaGetLastError();
}

}  // namespace gblu
