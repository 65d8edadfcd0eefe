// lpic_sort.cuh -- per-species counting sort by cell tile (Algorithm 1, "sort
// particles by cell index"), which also drops removed particles (the
// compaction of Sec. 2.1's lazy deletion).
//
// Three passes over the current buffer: histogram of tile keys (warp-
// aggregated atomics: neighbouring particles mostly share a tile), an
// exclusive scan of the ntiles+1 counts in one block, and a scatter into the
// other buffer.  Removed particles get key ntiles and are not written.  The
// order inside a tile follows atomic arrival and is not specified.
#pragma once
#include "lpic_common.cuh"
#include "lpic_fp32.cuh"
#include "lpic_fp64.cuh"

namespace lpic {

struct KeyFP32 {
    const int* cell;
    int nx, ny, T0, T1, T2, nt0, nt1, ntiles, dim;
    __device__ inline int operator()(int i) const {
        const int c = cell[i];
        if (c < 0) return ntiles;
        const int x = c % nx, r = c / nx, y = r % ny, z = (dim == 3) ? r / ny : 0;
        return ((z / T2) * nt1 + y / T1) * nt0 + x / T0;
    }
};

struct KeyFP64 {
    const double* x[3];
    const double* w;
    double rdx, rdy, rdz;
    int nx, ny, nz, T0, T1, T2, nt0, nt1, ntiles, dim;
    __device__ inline int operator()(int i) const {
        if (w[i] == 0.0) return ntiles;
        int cx = min(max((int)floor(x[0][i] * rdx), 0), nx - 1);
        int cy = min(max((int)floor(x[1][i] * rdy), 0), ny - 1);
        int cz = (dim == 3) ? min(max((int)floor(x[2][i] * rdz), 0), nz - 1) : 0;
        return ((cz / T2) * nt1 + cy / T1) * nt0 + cx / T0;
    }
};

__device__ inline unsigned lane_id() { return threadIdx.x & 31; }

template <class Key>
__global__ void k_sort_count(Key key, const int* n_ptr, int* count) {
    const int n = *n_ptr;
    const int stride = gridDim.x * blockDim.x;
    // every lane of a warp runs the same number of iterations
    const int nround = (n + stride - 1) / stride;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    for (int r = 0; r < nround; ++r, i += stride) {
        const bool valid = i < n;
        const int k = valid ? key(i) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, k);
        const int leader = __ffs(peers) - 1;
        if (valid && (int)lane_id() == leader) atomicAdd(count + k, __popc(peers));
    }
}

// Exclusive scan of count[0..len) into start[0..len], start[len] = total.
__global__ void k_sort_scan(const int* count, int* start, int len) {
    __shared__ int warp_sums[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < len; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int v = (i < len) ? count[i] : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if ((int)lane_id() >= o) x += y;
        }
        if (lane_id() == 31) warp_sums[threadIdx.x >> 5] = x;
        __syncthreads();
        if (threadIdx.x < 32) {
            const int nw = blockDim.x >> 5;
            int s = ((int)threadIdx.x < nw) ? warp_sums[threadIdx.x] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, s, o);
                if ((int)lane_id() >= o) s += y;
            }
            if ((int)threadIdx.x < nw) warp_sums[threadIdx.x] = s;
        }
        __syncthreads();
        const int wpre = (threadIdx.x >= 32) ? warp_sums[(threadIdx.x >> 5) - 1] : 0;
        if (i < len) start[i] = carry + wpre + x - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += wpre + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) start[len] = carry;
}

struct MoveFP32 {
    P32 src, dst;
    int dim;
    __device__ inline void operator()(int i, int j) const {
        dst.cell[j] = src.cell[i];
        dst.off[0][j] = src.off[0][i];
        dst.off[1][j] = src.off[1][i];
        if (dim == 3) dst.off[2][j] = src.off[2][i];
        dst.u[0][j] = src.u[0][i]; dst.u[1][j] = src.u[1][i]; dst.u[2][j] = src.u[2][i];
        dst.w[j] = src.w[i];
        dst.id[j] = src.id[i];
    }
};

struct MoveFP64 {
    P64 src, dst;
    int dim;
    __device__ inline void operator()(int i, int j) const {
        dst.x[0][j] = src.x[0][i];
        dst.x[1][j] = src.x[1][i];
        if (dim == 3) dst.x[2][j] = src.x[2][i];
        dst.u[0][j] = src.u[0][i]; dst.u[1][j] = src.u[1][i]; dst.u[2][j] = src.u[2][i];
        dst.w[j] = src.w[i];
        dst.id[j] = src.id[i];
    }
};

template <class Key, class Move>
__global__ void k_sort_scatter(Key key, Move mv, const int* n_ptr, const int* start, int* cursor,
                               int ntiles) {
    const int n = *n_ptr;
    const int stride = gridDim.x * blockDim.x;
    const int nround = (n + stride - 1) / stride;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    for (int r = 0; r < nround; ++r, i += stride) {
        const bool valid = i < n;
        const int k = valid ? key(i) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, k);
        const int leader = __ffs(peers) - 1;
        int base = 0;
        if (valid && (int)lane_id() == leader && k < ntiles) base = atomicAdd(cursor + k, __popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (valid && k < ntiles) {
            const int rank = __popc(peers & ((1u << lane_id()) - 1u));
            mv(i, start[k] + base + rank);
        }
    }
}

__global__ void k_sort_finalize(const int* start, int ntiles, int* n_out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *n_out = start[ntiles];
}

}  // namespace lpic
