// rx_order.cu -- spatial ordering of a batch's receivers.
//
// The class kernels take receivers in tiles of 32 consecutive ones; a tile
// whose receivers lie close together has small occluder masks (the
// receiver-side legs of body paths meet few bodies) and lanes that take the
// same branches.  Receivers that arrive in arbitrary order are therefore
// reordered per frame by a counting sort on the cells of a 128 x 128 grid over
// the scene's floor plan, the cells in Morton (Z) order:
//   1. count  -- each receiver's cell, and its rank among the receivers of
//                that cell (the value its atomic increment returned);
//   2. scan   -- per frame, the exclusive prefix sums of the cell counts;
//   3. place  -- receiver i goes to position offset(cell) + rank: the sorted
//                coordinates (SoA, per frame as the input) and, at that
//                position, i's index within its frame.
// Within a cell the order follows the atomics (it may differ from run to
// run); each receiver's fields do not depend on which receivers share its
// tile, so the outputs do not either.
#include "internal.h"

namespace creep {

namespace {

__device__ __forceinline__ uint32_t spread7(uint32_t v) {
    v &= 0x7fu;
    v = (v | (v << 4)) & 0x0f0fu;
    v = (v | (v << 2)) & 0x3333u;
    v = (v | (v << 1)) & 0x5555u;
    return v;
}

__device__ __forceinline__ uint32_t cell_of(float x, float y, const float4 g) {
    // g = (x0, y0, cells per metre in x, cells per metre in y)
    const float fx = fminf(fmaxf((x - g.x) * g.z, 0.0f), (float)(RX_GRID - 1));
    const float fy = fminf(fmaxf((y - g.y) * g.w, 0.0f), (float)(RX_GRID - 1));
    // (NaN coordinates land in cell 0)
    const uint32_t ix = (fx == fx) ? (uint32_t)fx : 0u, iy = (fy == fy) ? (uint32_t)fy : 0u;
    return spread7(ix) | (spread7(iy) << 1);
}

// grid: (blocks, n_frames); frame blockIdx.y
__global__ void k_rx_count(const FrameDev *__restrict__ frames, const float *__restrict__ rx, float4 g,
                           uint32_t *__restrict__ cnt, uint32_t *__restrict__ rank) {
    const FrameDev &F = frames[blockIdx.y];
    const float *x = rx + 3 * F.rx_off;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < F.n_rx; i += gridDim.x * blockDim.x) {
        const uint32_t c = cell_of(x[i], x[F.n_rx + i], g);
        rank[F.rx_off + i] = atomicAdd(&cnt[(size_t)blockIdx.y * RX_CELLS + c], 1u);
    }
}

// one block of 1024 threads per frame: exclusive scan of RX_CELLS counts in place
__global__ void __launch_bounds__(1024) k_rx_scan(uint32_t *__restrict__ cnt) {
    constexpr int PER = RX_CELLS / 1024;
    uint32_t *c = cnt + (size_t)blockIdx.x * RX_CELLS;
    __shared__ uint32_t s_sum[1024];
    uint32_t v[PER], run = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        v[k] = c[threadIdx.x * PER + k];
        run += v[k];
    }
    s_sum[threadIdx.x] = run;
    __syncthreads();
    // inclusive scan of the threads' sums (Hillis--Steele)
    for (int o = 1; o < 1024; o <<= 1) {
        const uint32_t add = threadIdx.x >= (unsigned)o ? s_sum[threadIdx.x - o] : 0u;
        __syncthreads();
        s_sum[threadIdx.x] += add;
        __syncthreads();
    }
    uint32_t off = threadIdx.x > 0 ? s_sum[threadIdx.x - 1] : 0u;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        c[threadIdx.x * PER + k] = off;
        off += v[k];
    }
}

__global__ void k_rx_place(const FrameDev *__restrict__ frames, const float *__restrict__ rx, float4 g,
                           const uint32_t *__restrict__ off, const uint32_t *__restrict__ rank,
                           float *__restrict__ rx_sorted, int32_t *__restrict__ perm) {
    const FrameDev &F = frames[blockIdx.y];
    const int n = F.n_rx;
    const float *x = rx + 3 * F.rx_off;
    float *y = rx_sorted + 3 * F.rx_off;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float px = x[i], py = x[n + i], pz = x[2 * n + i];
        const uint32_t c = cell_of(px, py, g);
        const uint32_t p = off[(size_t)blockIdx.y * RX_CELLS + c] + rank[F.rx_off + i];
        y[p] = px;
        y[n + p] = py;
        y[2 * n + p] = pz;
        perm[F.rx_off + p] = i;
    }
}

}  // namespace

int launch_rx_order(const FrameDev *frames_dev, int n_frames, int max_rx, const float *rx, float4 grid,
                    uint32_t *cnt, uint32_t *rank, float *rx_sorted, int32_t *perm, cudaStream_t st) {
    if (n_frames <= 0 || max_rx <= 0) return RT_OK;
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * (size_t)n_frames * RX_CELLS, st);
    const int blk = 256;
    int bx = (max_rx + blk - 1) / blk;
    if (bx > 64) bx = 64;
    if (n_frames > 65535) e = cudaErrorInvalidValue;
    if (e == cudaSuccess) {
        k_rx_count<<<dim3(bx, n_frames), blk, 0, st>>>(frames_dev, rx, grid, cnt, rank);
        k_rx_scan<<<n_frames, 1024, 0, st>>>(cnt);
        k_rx_place<<<dim3(bx, n_frames), blk, 0, st>>>(frames_dev, rx, grid, cnt, rank, rx_sorted, perm);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_error(std::string("receiver ordering: ") + cudaGetErrorString(e));
        return RT_ERR_CUDA;
    }
    return RT_OK;
}

}  // namespace creep
