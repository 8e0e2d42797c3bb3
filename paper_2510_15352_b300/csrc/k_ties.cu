// k_ties.cu -- the tie-break of the depth order.
//
// The method orders a tile's Gaussians by depth and, at equal depth, by the
// Gaussian's index. The projection writes a camera's survivors in the
// library's storage order (spatial, see k_scene.cu) and the depth sort is
// stable, so equal keys leave the sort in storage order. This pass restores
// the index order: within every run of equal keys of a segment it reorders the
// run's values (slots) by the caller's index of their Gaussians, oidx[seg_base
// + slot] (written by the projection).
//
// Equal float32 depths are common (hundreds of pairs per full-size camera);
// long runs are not (many Gaussians at exactly one depth, such as a plane
// facing the camera). The thread that finds the start of a run of up to 32
// entries reorders it in place by insertion; longer runs are listed and each
// is sorted by one block: a stable LSD radix sort of (index, slot) pairs, 8
// bits per pass, ping-ponging through the depth sort's other buffers (free
// once the sort is done). The keys of a run are all equal, so their array
// holds the indices during the block sort and gets the key back at the end.
#include "gs_internal.cuh"

namespace gsk {

namespace {

constexpr int TT = 256;        // threads per detection block
constexpr int TPT = 8;         // keys per thread: one 2048-key sort tile per block pass
constexpr int SHORT = 32;      // runs up to this length are reordered in place
constexpr int LT = 1024;       // threads per long-run block
constexpr int LW = LT / 32;

struct TieRun {
    long long start;     // first position of the run in keys / vals
    long long seg_base;  // first position of its segment
    int len, pad;
};

// Sorts a run of equal keys [j, j + L) of the segment at base by the caller index.
__device__ __noinline__ void order_run(uint32_t *__restrict__ vals, const uint32_t *__restrict__ oidx,
                                       long long base, int j, int L, TieRun *__restrict__ runs,
                                       long long capacity, int *__restrict__ n_runs) {
    if (L <= SHORT) {
        uint32_t *v = vals + base + j;
        uint32_t sv[SHORT], so[SHORT];
        for (int i = 0; i < L; ++i) {
            sv[i] = v[i];
            so[i] = oidx[base + sv[i]];
        }
        for (int i = 1; i < L; ++i) {  // insertion by index (indices are distinct)
            const uint32_t a = so[i], b = sv[i];
            int t = i - 1;
            while (t >= 0 && so[t] > a) {
                so[t + 1] = so[t];
                sv[t + 1] = sv[t];
                --t;
            }
            so[t + 1] = a;
            sv[t + 1] = b;
        }
        for (int i = 0; i < L; ++i) v[i] = sv[i];
    } else {
        const int r = atomicAdd(n_runs, 1);
        if (r < capacity) runs[r] = TieRun{base + j, base, L, 0};
    }
}

// One sort tile (2,048 keys) per block pass; thread t looks at the TPT
// consecutive keys from t0 + TPT t, loaded together with the key before them
// and the one after (the lanes' loads are issued at once, not one by one).
__global__ void __launch_bounds__(TT)
    k_tie_detect(const uint32_t *__restrict__ keys, uint32_t *__restrict__ vals,
                 const uint32_t *__restrict__ oidx, const SortTile *__restrict__ tiles,
                 const int *__restrict__ n_tiles_dev, TieRun *__restrict__ runs,
                 long long capacity, int *__restrict__ n_runs) {
    const int nt = *n_tiles_dev;
    for (int tile = blockIdx.x; tile < nt; tile += gridDim.x) {
        const SortTile T = tiles[tile];
        const uint32_t *k = keys + T.seg_base;
        const int j0 = T.t0 + TPT * (int)threadIdx.x;
        const int end = T.t0 + T.nk;
        if (j0 >= end) continue;
        uint32_t kv[TPT + 2];  // keys j0 - 1 .. j0 + TPT (0xffffffff... outside the segment)
#pragma unroll
        for (int q = 0; q < TPT + 2; ++q) {
            const int j = j0 - 1 + q;
            kv[q] = (j >= 0 && j < T.seg_n) ? k[j] : (q == 0 ? 0xfffffffeu : 0xffffffffu);
        }
        // a run starts at j when k[j] == k[j + 1] and (j is the first or k[j - 1] != k[j]);
        // the sentinels differ from each other, so no run starts past the segment
        uint32_t starts = 0u;
#pragma unroll
        for (int q = 1; q <= TPT; ++q)
            if (j0 - 1 + q < end && kv[q] == kv[q + 1] && kv[q - 1] != kv[q]) starts |= 1u << q;
        while (starts) {
            const int q = __ffs(starts) - 1;
            starts &= starts - 1u;
            const int j = j0 - 1 + q;
            const uint32_t kj = kv[q];
            int e = j + 2;
            while (e < T.seg_n && k[e] == kj) ++e;
            order_run(vals, oidx, T.seg_base, j, e - j, runs, capacity, n_runs);
        }
    }
}

__global__ void __launch_bounds__(LT)
    k_tie_long(uint32_t *__restrict__ keys, uint32_t *__restrict__ vals,
               uint32_t *__restrict__ sk, uint32_t *__restrict__ sv,
               const uint32_t *__restrict__ oidx, const TieRun *__restrict__ runs,
               long long capacity, const int *__restrict__ n_runs) {
    __shared__ int wcnt[LW][256 + 1];  // per warp and digit (+1: the idle lanes' digit)
    __shared__ int off[256];
    __shared__ uint32_t red[LW];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const long long nr = min((long long)*n_runs, capacity);
    for (long long r = blockIdx.x; r < nr; r += gridDim.x) {
        const TieRun R = runs[r];
        const int L = R.len;
        uint32_t *AK = keys + R.start, *AV = vals + R.start;
        uint32_t *BK = sk + R.start, *BV = sv + R.start;
        const uint32_t kz = AK[0];
        __syncthreads();  // every thread has read kz before it is overwritten
        uint32_t mx = 0;
        for (int i = tid; i < L; i += LT) {
            const uint32_t o = oidx[R.seg_base + AV[i]];
            AK[i] = o;
            mx = max(mx, o);
        }
        for (int i = tid; i < LW * 257; i += LT) (&wcnt[0][0])[i] = 0;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, d));
        if (lane == 0) red[warp] = mx;
        __syncthreads();
        mx = 0;
        for (int w = 0; w < LW; ++w) mx = max(mx, red[w]);
        int passes = 1;
        while (passes < 4 && (mx >> (8 * passes)) != 0u) ++passes;
        uint32_t *srcK = AK, *srcV = AV, *dstK = BK, *dstV = BV;
        for (int p = 0; p < passes; ++p) {
            const int sh = 8 * p;
            if (tid < 256) off[tid] = 0;
            __syncthreads();
            for (int i = tid; i < L; i += LT) atomicAdd(&off[(srcK[i] >> sh) & 255u], 1);
            __syncthreads();
            if (warp == 0) {  // exclusive prefix of the 256 counts, 8 per lane
                int v[8], s = 0;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    v[q] = off[8 * lane + q];
                    s += v[q];
                }
                int incl = s;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const int t = __shfl_up_sync(0xffffffffu, incl, d);
                    if (lane >= d) incl += t;
                }
                int run = incl - s;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    off[8 * lane + q] = run;
                    run += v[q];
                }
            }
            __syncthreads();
            for (int base = 0; base < L; base += LT) {
                const int i = base + tid;
                const bool valid = i < L;
                const uint32_t key = valid ? srcK[i] : 0u, val = valid ? srcV[i] : 0u;
                const int d = valid ? (int)((key >> sh) & 255u) : 256;
                const uint32_t peers = __match_any_sync(0xffffffffu, d);
                const int rank = __popc(peers & lt);
                if (rank == 0) wcnt[warp][d] = __popc(peers);
                __syncthreads();
                if (valid) {
                    int pos = off[d] + rank;
                    for (int w = 0; w < warp; ++w) pos += wcnt[w][d];
                    dstK[pos] = key;
                    dstV[pos] = val;
                }
                __syncthreads();
                if (tid < 256) {
                    int s = 0;
                    for (int w = 0; w < LW; ++w) {
                        s += wcnt[w][tid];
                        wcnt[w][tid] = 0;
                    }
                    off[tid] += s;
                } else if (tid < 256 + LW) {
                    wcnt[tid - 256][256] = 0;
                }
                __syncthreads();
            }
            uint32_t *t = srcK;
            srcK = dstK;
            dstK = t;
            t = srcV;
            srcV = dstV;
            dstV = t;
        }
        // the sorted run is in src; values back to vals, the key back to keys
        for (int i = tid; i < L; i += LT) {
            if (srcV != AV) AV[i] = srcV[i];
            AK[i] = kz;
        }
        __syncthreads();
    }
}

}  // namespace

size_t tie_run_bytes() { return sizeof(TieRun); }

cudaError_t launch_tie_order(uint32_t *keys, uint32_t *vals, uint32_t *scratch_k,
                             uint32_t *scratch_v, const uint32_t *oidx, const SortTile *tiles,
                             const int *n_tiles_dev, int grid, void *runs, long long capacity,
                             int *n_runs, cudaStream_t s) {
    k_tie_detect<<<grid, TT, 0, s>>>(keys, vals, oidx, tiles, n_tiles_dev, (TieRun *)runs,
                                     capacity, n_runs);
    k_tie_long<<<148, LT, 0, s>>>(keys, vals, scratch_k, scratch_v, oidx, (const TieRun *)runs,
                                  capacity, n_runs);
    return cudaGetLastError();
}

}  // namespace gsk
