// gs_noalloc.cu -- the segmented sort for callers that cannot allocate GPU
// memory.
//
// Some callers cannot call cudaMalloc: code running inside a CUDA graph or a
// stream-ordered region they do not own, plugins whose host application owns
// every device allocation (a simulator that pre-reserves all GPU memory for
// its physics and gives extensions only the buffers it hands them), or
// real-time loops that forbid allocation after start-up. gs_sort_segments
// needs a context whose workspace grows with cudaMalloc; this entry point does
// the same sort with its scratch in a fixed file-scope device array instead.
//
// The scratch is a static __device__ array of GS_NOALLOC_SCRATCH_BYTES: every
// GPU that loads this library holds it until the process exits. Host code
// cannot use the array's name as a device address (on the host it names a
// host-side shadow), so on the first call on each device, with that device
// current, the device address is looked up once with cudaGetSymbolAddress and
// cached. That first call therefore makes a CUDA runtime query: issue it
// before any stream capture. All calls share the one array and it keeps the
// last call's contents; calls whose work overlaps on the GPU (two streams, or
// two host threads) race on it and must be serialised by the caller.
#include <mutex>

#include "gs.h"
#include "gs_internal.cuh"

namespace {

using namespace gsk;

constexpr long long NA_MAX_KEYS = 1LL << 21;  // keys per call
constexpr int NA_MAX_SEGS = 4096;             // segments per call
constexpr int NA_TK = 2048;                   // keys per sort tile (matches k_sort.cu)
constexpr long long NA_MAX_TILES = NA_MAX_KEYS / NA_TK + NA_MAX_SEGS;

// scratch layout (in 4-byte words)
constexpr long long OFF_TKEYS = 0;
constexpr long long OFF_TVALS = OFF_TKEYS + NA_MAX_KEYS;
constexpr long long OFF_HIST = OFF_TVALS + NA_MAX_KEYS;
constexpr long long OFF_TILES = OFF_HIST + NA_MAX_TILES * 256;
constexpr long long OFF_SEGS = OFF_TILES + NA_MAX_SEGS + 8;  // 2 * NA_MAX_SEGS int64, 8-aligned
constexpr long long SCRATCH_WORDS = OFF_SEGS + 4LL * NA_MAX_SEGS;

static __device__ __align__(256) uint32_t g_noalloc_scratch[SCRATCH_WORDS];

// Per segment: a validated copy of (start, count) -- a segment outside
// [0, n) is treated as empty -- and the prefix of its sort-tile counts.
__global__ void __launch_bounds__(1024)
    k_noalloc_tiles(const int64_t *__restrict__ seg_start, const int64_t *__restrict__ seg_count,
                    int n_seg, long long n, long long *__restrict__ vstart,
                    long long *__restrict__ vcount, int *__restrict__ tile_start) {
    __shared__ int wsum[32];
    __shared__ int carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int b = 0; b < n_seg; b += 1024) {
        const int i = b + tid;
        int tiles = 0;
        if (i < n_seg) {
            long long s = seg_start[i], c = seg_count[i];
            if (s < 0 || c < 0 || s > n || c > n - s) c = 0;
            if (s < 0 || s > n) s = 0;
            vstart[i] = s;
            vcount[i] = c;
            tiles = (int)((c + NA_TK - 1) / NA_TK);
        }
        int incl = tiles;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += v;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < 32; ++w) {
            const int v = wsum[w];
            before += w < warp ? v : 0;
            total += v;
        }
        if (i < n_seg) tile_start[i] = carry + before + incl - tiles;
        __syncthreads();
        if (tid == 0) carry += total;
        __syncthreads();
    }
    if (tid == 0) tile_start[n_seg] = carry;
}

std::mutex g_setup_mutex;
uint32_t *g_scratch_ptr[64] = {};  // device address of the scratch, per device

}  // namespace

extern "C" gs_status gs_sort_segments_noalloc(uint32_t *keys, uint32_t *vals, int64_t n,
                                              const int64_t *seg_start,
                                              const int64_t *seg_count, int32_t n_seg,
                                              void *stream) {
    if (n < 0 || n_seg < 0) return GS_ERR_INVALID_ARG;
    if (n > NA_MAX_KEYS || n_seg > NA_MAX_SEGS) return GS_ERR_CAPACITY;
    if (n_seg == 0 || n == 0) return GS_OK;
    if (!keys || !vals || !seg_start || !seg_count) return GS_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return GS_ERR_CUDA;
    uint32_t *base;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p)
                return GS_ERR_CUDA;
            g_scratch_ptr[dev] = (uint32_t *)p;
        }
        base = g_scratch_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    long long *vstart = (long long *)(base + OFF_SEGS);
    long long *vcount = vstart + NA_MAX_SEGS;
    int *tiles = (int *)(base + OFF_TILES);
    k_noalloc_tiles<<<1, 1024, 0, st>>>(seg_start, seg_count, n_seg, n, vstart, vcount, tiles);
    if (cudaGetLastError() != cudaSuccess) return GS_ERR_CUDA;
    // grid for the largest possible tile count; tiles past the real total
    // find no keys and write nothing
    const int tiles_upper = (int)((n + NA_TK - 1) / NA_TK) + n_seg;
    if (launch_sort_segments(keys, vals, base + OFF_TKEYS, base + OFF_TVALS, vstart, vcount, tiles,
                             n_seg, tiles_upper, base + OFF_HIST, st) != cudaSuccess)
        return GS_ERR_CUDA;
    return GS_OK;
}
