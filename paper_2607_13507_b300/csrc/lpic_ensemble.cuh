// lpic_ensemble.cuh -- batched kernels for an ensemble of independent grids
// stepped together: one launch per field pass and per sort pass covers every
// grid (blockIdx.y = grid or species slot), and one persistent particle kernel
// (k_gpd32_queue) pulls (slot, work item) entries from a device queue.
#pragma once
#include "lpic_common.cuh"
#include "lpic_field.cuh"
#include "lpic_fp32.cuh"
#include "lpic_sort.cuh"

namespace lpic {

struct EnsField {
    Geo g;
    FieldArgs<float, long long> a;
    unsigned long long* J[3];
    long long nfield;
};

struct EnsSort {
    KeyFP32 key[2];          // keys reading buffer 0 / buffer 1
    MoveFP32 mv[2];          // moves from buffer p to buffer 1 - p
    int* n;                  // particles in the current buffer
    int* count;
    int* start;
    int* cursor;
    int* coff;
    int2* items;
    int* nitems;
    int* nesc;
    int ntiles, P;
};

template <int DIM>
__global__ void k_update_E_many(const EnsField* f) {
    const EnsField& F = f[blockIdx.y];
    update_E_range<DIM>(F.g, F.a, blockIdx.x * (long long)blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
}

template <int DIM>
__global__ void k_update_B_many(const EnsField* f) {
    const EnsField& F = f[blockIdx.y];
    update_B_range<DIM>(F.g, F.a, blockIdx.x * (long long)blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
}

static __global__ void k_zero_J_many(const EnsField* f) {
    const EnsField& F = f[blockIdx.y];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < F.nfield;
         i += (long long)gridDim.x * blockDim.x) {
        F.J[0][i] = 0; F.J[1][i] = 0; F.J[2][i] = 0;
    }
}

// cursors (and, on request, the histograms) to zero; escape counters to zero
static __global__ void k_sort_zero_many(const EnsSort* s, int zero_count) {
    const EnsSort& S = s[blockIdx.y];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= S.ntiles; i += gridDim.x * blockDim.x) {
        S.cursor[i] = 0;
        if (zero_count) S.count[i] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *S.nesc = 0;
}

static __global__ void k_count_zero_many(const EnsSort* s) {
    const EnsSort& S = s[blockIdx.y];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= S.ntiles; i += gridDim.x * blockDim.x) S.count[i] = 0;
}

static __global__ void k_sort_count_many(const EnsSort* s, int parity) {
    const EnsSort& S = s[blockIdx.y];
    sort_count_body(S.key[parity], *S.n, S.count, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

static __global__ void k_sort_scan_many(const EnsSort* s) {
    const EnsSort& S = s[blockIdx.x];
    const int* count = S.count;
    const int P = S.P;
    block_scan([count](int i) { return count[i]; }, S.start, S.ntiles + 1);
    block_scan([count, P](int i) { return (count[i] + P - 1) / P; }, S.coff, S.ntiles);
}

static __global__ void k_sort_items_many(const EnsSort* s) {
    const EnsSort& S = s[blockIdx.y];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < S.ntiles; t += gridDim.x * blockDim.x) {
        const int nch = (S.count[t] + S.P - 1) / S.P;
        const int o = S.coff[t];
        for (int c = 0; c < nch; ++c) S.items[o + c] = make_int2(t, c);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *S.nitems = S.coff[S.ntiles];
}

static __global__ void k_sort_scatter_many(const EnsSort* s, int parity) {
    const EnsSort& S = s[blockIdx.y];
    sort_scatter_body(S.key[parity], S.mv[parity], *S.n, S.start, S.cursor, S.ntiles,
                      blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

static __global__ void k_sort_finalize_many(const EnsSort* s, int nslots) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nslots; i += gridDim.x * blockDim.x)
        *s[i].n = s[i].start[s[i].ntiles];
}

// Queue offsets of the slots in processing order; resets the queue head.
static __global__ void k_queue_prefix(const EnsSort* s, const int* order, int nslots, int* prefix, int* head) {
    block_scan([s, order](int r) { return *s[order[r]].nitems; }, prefix, nslots);
    if (threadIdx.x == 0) *head = 0;
}

// Sets bit LPIC_ST_HALO if any particle was queued for the global-memory path
// (cannot happen while the ensemble sorts every step).
static __global__ void k_check_escapes(const EnsSort* s, int nslots, unsigned* st) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nslots; i += gridDim.x * blockDim.x)
        if (*s[i].nesc != 0) atomicOr(st, LPIC_ST_HALO);
}

}  // namespace lpic
