// lpic_noalloc.cu -- a tile sort that needs no allocation from its caller or
// from the library.
//
// lpic_sort_particles needs a grid, and creating a grid allocates scratch with
// cudaMalloc.  Some callers cannot do that: a host framework that owns all
// device memory through its own pool (and forbids the CUDA allocator), code
// that runs while another thread is capturing a CUDA graph in global capture
// mode (where cudaMalloc is an illegal call), or a real-time loop that cannot
// afford the implicit device synchronisation of cudaMalloc/cudaFree.  For
// them this file provides the same counting sort by cell tile over a caller's
// FP32 particle buffer, with its scratch (tile histogram, offsets, cursors) in
// one fixed-size array in device global memory that lives for as long as the
// library is loaded.
//
// In host code the array's name only stands for the symbol; the kernels get
// its device address, looked up once per device with cudaGetSymbolAddress.
#include <cstring>
#include <mutex>

#include "lpic.h"
#include "lpic_common.cuh"
#include "lpic_fp32.cuh"
#include "lpic_sort.cuh"

using namespace lpic;

namespace lpic {
void set_last_error(const char* msg);   // lpic_last_error() reports it
}

namespace {

constexpr int kMaxTiles = LPIC_NOALLOC_MAX_TILES;
// histogram (ntiles + 1), scan output (ntiles + 2), cursors (ntiles + 1),
// work-item offsets (ntiles + 1), then the particle count actually sorted;
// each part starts on a 256-byte boundary.
constexpr int kPart = (kMaxTiles + 2 + 63) / 64 * 64;
static __device__ __align__(256) int lpic_noalloc_scratch[4 * kPart + 64];

std::mutex g_mu;
int* g_scratch[64] = {nullptr};
int g_nsm[64] = {0};

lpic_status nfail(lpic_status s, const char* m) {
    set_last_error(m);
    return s;
}

// Device address of the scratch array and the SM count of the current
// device; the first call on a device looks both up (so that first call must
// not happen while the calling thread captures a graph).
lpic_status scratch_ptr(int** out, int* nsm) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return nfail(LPIC_ECUDA, "lpic_sort_tiles_static: no current CUDA device");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, lpic_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return nfail(LPIC_ECUDA, "lpic_sort_tiles_static: cudaGetSymbolAddress failed");
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
            return nfail(LPIC_ECUDA, "lpic_sort_tiles_static: cannot query the SM count");
        g_nsm[dev] = n;
        g_scratch[dev] = static_cast<int*>(p);
    }
    *out = g_scratch[dev];
    *nsm = g_nsm[dev];
    return LPIC_OK;
}

// Tile key of a caller's particle: cells outside [0, ncells) are treated as
// removed (key ntiles), like cell < 0, so that no histogram entry outside the
// scratch array is touched.
struct KeyChecked {
    KeyFP32 key;
    int ncells;
    __device__ inline int operator()(int i) const {
        const int c = key.cell[i];
        return (c >= ncells) ? key.ntiles : key(i);
    }
};

// The number of particles sorted: the caller's count, clamped to [0, capacity].
__global__ void k_clamp_count(const int* count_in, long long capacity, int* n) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const int c = *count_in;
        *n = c < 0 ? 0 : (c > capacity ? (int)capacity : c);
    }
}

P32 view(void* buf, long long cap, int dim, const int* n) {
    char* base = static_cast<char*>(buf);
    const size_t a = (size_t)cap * 4;
    P32 p{};
    p.cell = reinterpret_cast<int*>(base);
    for (int d = 0; d < 3; ++d) p.off[d] = reinterpret_cast<float*>(base + (1 + (d < dim ? d : dim - 1)) * a);
    for (int c = 0; c < 3; ++c) p.u[c] = reinterpret_cast<float*>(base + (1 + dim + c) * a);
    p.w = reinterpret_cast<float*>(base + (4 + dim) * a);
    p.id = reinterpret_cast<int*>(base + (5 + dim) * a);
    p.n = n;
    return p;
}

__global__ void k_copy_starts(const int* start, int* out, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = start[i];
}

}  // namespace

extern "C" lpic_status lpic_sort_tiles_static(int dim, int nx, int ny, int nz, const int tile[3],
                                              const void* src, void* dst, long long capacity,
                                              const int* count_in, int* count_out,
                                              int* tile_start, cudaStream_t stream) {
    if (dim != 2 && dim != 3) return nfail(LPIC_EINVAL, "lpic_sort_tiles_static: dim must be 2 or 3");
    if (dim == 2) nz = 1;
    if (nx < 1 || ny < 1 || nz < 1 || (long long)nx * ny * nz >= (1LL << 31))
        return nfail(LPIC_EINVAL, "lpic_sort_tiles_static: bad grid size");
    if (!tile) return nfail(LPIC_EINVAL, "lpic_sort_tiles_static: tile is NULL");
    int T[3] = {tile[0], tile[1], dim == 3 ? tile[2] : 1};
    const int n3[3] = {nx, ny, nz};
    long long ntiles = 1;
    int nt[3];
    for (int k = 0; k < 3; ++k) {
        if (T[k] < 1 || T[k] > n3[k]) return nfail(LPIC_EINVAL, "lpic_sort_tiles_static: tile size out of range");
        nt[k] = (n3[k] + T[k] - 1) / T[k];
        ntiles *= nt[k];
    }
    if (ntiles > kMaxTiles)
        return nfail(LPIC_EINVAL, "lpic_sort_tiles_static: more tiles than LPIC_NOALLOC_MAX_TILES");
    if (!src || !dst || src == dst || !count_in || !count_out || !tile_start)
        return nfail(LPIC_EINVAL, "lpic_sort_tiles_static: NULL or aliased pointer");
    if (capacity <= 0 || capacity % 64 != 0 || capacity >= (1LL << 31))
        return nfail(LPIC_EINVAL, "lpic_sort_tiles_static: capacity must be a positive multiple of 64 below 2^31");
    if ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) % 256 != 0)
        return nfail(LPIC_EINVAL, "lpic_sort_tiles_static: buffers must be 256-byte aligned");

    int* scratch = nullptr;
    int nsm = 0;
    if (lpic_status r = scratch_ptr(&scratch, &nsm)) return r;
    int* count = scratch;
    int* start = scratch + kPart;
    int* cursor = scratch + 2 * kPart;
    int* coff = scratch + 3 * kPart;
    int* n_sorted = scratch + 4 * kPart;
    const int nt1 = (int)ntiles;
    // the array keeps the previous call's contents: clear what must start at zero
    if (cudaMemsetAsync(count, 0, sizeof(int) * (nt1 + 1), stream) != cudaSuccess ||
        cudaMemsetAsync(cursor, 0, sizeof(int) * (nt1 + 1), stream) != cudaSuccess)
        return nfail(LPIC_ECUDA, "lpic_sort_tiles_static: cudaMemsetAsync failed");

    const P32 s = view(const_cast<void*>(src), capacity, dim, n_sorted);
    const P32 d = view(dst, capacity, dim, count_out);
    const CellDecode dec{make_fastdiv((unsigned)nx), make_fastdiv((unsigned)ny)};
    const KeyChecked key{KeyFP32{s.cell, dec, make_fastdiv((unsigned)T[0]), make_fastdiv((unsigned)T[1]),
                                 make_fastdiv((unsigned)T[2]), nt[0], nt[1], nt1},
                         nx * ny * nz};
    // grid-stride kernels: at most 16 blocks of 256 per SM
    int blocks = (int)((capacity + 255) / 256);
    if (blocks > nsm * 16) blocks = nsm * 16;
    k_clamp_count<<<1, 32, 0, stream>>>(count_in, capacity, n_sorted);
    k_sort_count<<<blocks, 256, 0, stream>>>(key, n_sorted, count);
    k_sort_scan<<<1, 1024, 0, stream>>>(count, start, nt1, 1 << 30, coff);
    k_sort_scatter<<<blocks, 256, 0, stream>>>(key, MoveFP32{s, d, dim}, n_sorted, start, cursor, nt1);
    k_sort_finalize<<<1, 32, 0, stream>>>(start, nt1, count_out);
    k_copy_starts<<<(nt1 + 1 + 255) / 256, 256, 0, stream>>>(start, tile_start, nt1 + 1);
    if (cudaGetLastError() != cudaSuccess) return nfail(LPIC_ECUDA, "lpic_sort_tiles_static: kernel launch failed");
    return LPIC_OK;
}
