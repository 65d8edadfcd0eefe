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
    CellDecode dec;
    FastDiv T0, T1, T2;
    int nt0, nt1, ntiles;
    __device__ inline int operator()(int i) const {
        const int c = cell[i];
        if (c < 0) return ntiles;
        int gc[3];
        dec(c, gc);
        return (fdiv(gc[2], T2) * nt1 + fdiv(gc[1], T1)) * nt0 + fdiv(gc[0], T0);
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
__device__ inline void sort_count_body(const Key& key, int n, int* count, int i, int stride) {
    // every lane of a warp runs the same number of iterations
    const int nround = (n + stride - 1) / stride;
    for (int r = 0; r < nround; ++r, i += stride) {
        const bool valid = i < n;
        const int k = valid ? key(i) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, k);
        const int leader = __ffs(peers) - 1;
        if (valid && (int)lane_id() == leader) atomicAdd(count + k, __popc(peers));
    }
}

template <class Key>
__global__ void k_sort_count(Key key, const int* n_ptr, int* count) {
    sort_count_body(key, *n_ptr, count, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// Exclusive block-wide scan of f(0..len) into out[0..len], out[len] = total.
template <class F>
__device__ inline void block_scan(F f, int* out, int len) {
    __shared__ int warp_sums[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < len; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int v = (i < len) ? f(i) : 0;
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
        if (i < len) out[i] = carry + wpre + x - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += wpre + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) out[len] = carry;
    __syncthreads();
}

// start = exclusive scan of the ntiles + 1 key counts (the last key holds
// removed particles); coff = exclusive scan of the work-item counts
// ceil(count / P) of the ntiles tiles, coff[ntiles] = number of items.
static __global__ void k_sort_scan(const int* count, int* start, int ntiles, int P, int* coff) {
    block_scan([count](int i) { return count[i]; }, start, ntiles + 1);
    block_scan([count, P](int i) { return (count[i] + P - 1) / P; }, coff, ntiles);
}

// Work items (tile, chunk), tile-major.
static __global__ void k_sort_items(const int* count, const int* coff, int ntiles, int P, int2* items,
                             int* nitems) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += gridDim.x * blockDim.x) {
        const int nch = (count[t] + P - 1) / P;
        const int o = coff[t];
        for (int c = 0; c < nch; ++c) items[o + c] = make_int2(t, c);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *nitems = coff[ntiles];
}

// A particle's record: load() reads it (before the destination is known, so
// the loads overlap the cursor atomic), store() writes it.
struct MoveFP32 {
    P32 src, dst;
    int dim;
    struct Rec { int cell, id; float off[3], u[3], w; };
    __device__ inline Rec load(int i) const {
        Rec r;
        r.cell = src.cell[i];
        r.off[0] = src.off[0][i];
        r.off[1] = src.off[1][i];
        r.off[2] = (dim == 3) ? src.off[2][i] : 0.0f;
        r.u[0] = src.u[0][i]; r.u[1] = src.u[1][i]; r.u[2] = src.u[2][i];
        r.w = src.w[i];
        r.id = src.id[i];
        return r;
    }
    __device__ inline void store(const Rec& r, int j) const {
        dst.cell[j] = r.cell;
        dst.off[0][j] = r.off[0];
        dst.off[1][j] = r.off[1];
        if (dim == 3) dst.off[2][j] = r.off[2];
        dst.u[0][j] = r.u[0]; dst.u[1][j] = r.u[1]; dst.u[2][j] = r.u[2];
        dst.w[j] = r.w;
        dst.id[j] = r.id;
    }
};

struct MoveFP64 {
    P64 src, dst;
    int dim;
    struct Rec { double x[3], u[3], w; int id; };
    __device__ inline Rec load(int i) const {
        Rec r;
        r.x[0] = src.x[0][i];
        r.x[1] = src.x[1][i];
        r.x[2] = (dim == 3) ? src.x[2][i] : 0.0;
        r.u[0] = src.u[0][i]; r.u[1] = src.u[1][i]; r.u[2] = src.u[2][i];
        r.w = src.w[i];
        r.id = src.id[i];
        return r;
    }
    __device__ inline void store(const Rec& r, int j) const {
        dst.x[0][j] = r.x[0];
        dst.x[1][j] = r.x[1];
        if (dim == 3) dst.x[2][j] = r.x[2];
        dst.u[0][j] = r.u[0]; dst.u[1][j] = r.u[1]; dst.u[2][j] = r.u[2];
        dst.w[j] = r.w;
        dst.id[j] = r.id;
    }
};

template <class Key, class Move>
__device__ inline void sort_scatter_body(const Key& key, const Move& mv, int n, const int* start,
                                         int* cursor, int ntiles, int i, int stride) {
    const int nround = (n + stride - 1) / stride;
    for (int r = 0; r < nround; ++r, i += stride) {
        const bool valid = i < n;
        const int k = valid ? key(i) : -1;
        typename Move::Rec rec{};
        if (valid && k < ntiles) rec = mv.load(i);
        const unsigned peers = __match_any_sync(0xffffffffu, k);
        const int leader = __ffs(peers) - 1;
        int base = 0;
        if (valid && (int)lane_id() == leader && k < ntiles) base = atomicAdd(cursor + k, __popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (valid && k < ntiles) {
            const int rank = __popc(peers & ((1u << lane_id()) - 1u));
            mv.store(rec, start[k] + base + rank);
        }
    }
}

template <class Key, class Move>
__global__ void k_sort_scatter(Key key, Move mv, const int* n_ptr, const int* start, int* cursor,
                               int ntiles) {
    sort_scatter_body(key, mv, *n_ptr, start, cursor, ntiles, blockIdx.x * blockDim.x + threadIdx.x,
                      gridDim.x * blockDim.x);
}

static __global__ void k_sort_finalize(const int* start, int ntiles, int* n_out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *n_out = start[ntiles];
}

}  // namespace lpic
