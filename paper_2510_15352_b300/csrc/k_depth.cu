// k_depth.cu -- the render's depth order: every camera's survivors sorted by
// (depth, caller index of the Gaussian), the order in which a tile is
// composited front to back (Sec. 3.2 of the paper renders with the 3DGS
// rasteriser, which orders a tile's Gaussians by view-space depth; equal depths
// go in index order).
//
// Input: per camera (segment) the survivors' depth keys in slot order, key =
// bits(z) - bits(near) (monotone in z, non-negative for z > near). Output: keys
// and slots in that order. The tie-break is a total order (the caller indices
// of a camera's survivors are distinct), so no step needs to be stable:
//
//   k_depth_count   per camera, how many keys fall in each of 2,048 buckets (key
//                   bits 15-25; keys of 2^26 or more all in the last bucket): a
//                   shared-memory histogram per 2,048-key sort tile, then one
//                   global atomic per non-empty bucket of the tile;
//   k_depth_scan    per camera: bucket starts (the scatter's cursors) and the
//                   windows: window w owns the buckets that start at positions
//                   [1024 w, 1024 w + 1024) and covers exactly those buckets;
//   k_depth_scatter each tile grouped by bucket in shared memory, its share of
//                   every bucket reserved with one global atomic on the bucket's
//                   cursor (after the pass, the cursor is the bucket's end), then
//                   written out run by run (key and slot);
//   k_depth_window  each window sorted in shared memory by a block of 256
//                   threads: a counting sort in which a bucket of c keys gets c
//                   bins (by the key's low bits), then each key's rank inside its
//                   bin (equal keys by staged position); the slots are written
//                   back and every run of equal keys is listed. The next window
//                   is copied in (cp.async) while one is sorted. A window of
//                   more than 2,048 keys, over more than 512 buckets, or with a
//                   bin of more than 32 keys is listed instead;
//   k_depth_big     a listed window sorted by one block (stable LSD radix sort,
//                   8 bits per pass, in shared memory up to 4,096 keys, else
//                   through global scratch), then its runs of equal keys put in
//                   caller-index order (short runs in place, longer ones listed);
//   k_tie_long      a listed run of more than 32 equal keys sorted by caller
//                   index, one block;
//   k_tie_short     the runs of equal keys the window pass listed, one thread
//                   each: slots in caller-index order.
//
// A bucket is 1/256 of the depth; on the full-size workloads the largest hold
// about 1,400 keys, so windows average 1,024 keys and few pass 2,048 (about one
// per camera goes to k_depth_big; 512-position windows averaged 2.5 keys per
// thread, and the per-window costs made the window pass 14 % slower). Equal float32 depths are common: about
// 1,800 runs per camera, nearly all pairs. Nothing after the depth order reads
// the sorted keys, so only the windows listed for the block sort keep theirs
// up to date.
#include <algorithm>

#include "gs_internal.cuh"

namespace gsk {

namespace {

constexpr int NB = DEPTH_BUCKETS;          // buckets per camera (2048)
constexpr int BSH = 15;                    // a key's bucket: key >> BSH (clamped)
constexpr int BT = 256;                    // threads of the count / scatter blocks
constexpr int BPT = SORT_TILE_KEYS / BT;   // keys per thread (8)
constexpr int WIN = DEPTH_WINDOW;          // window stride (1024)
constexpr int WPS = SORT_TILE_KEYS / WIN;  // windows per sort tile (2)
constexpr int WT = 256;                    // threads per window block
constexpr int WPT = 8;                     // keys per thread of a window block
constexpr int WCAP = WT * WPT;             // largest window sorted in shared memory (2048)
constexpr int BIN_MAX = 32;                // largest bin the window pass ranks (else: block sort)
constexpr int SHORT = 32;                  // runs up to this length are ordered in place
constexpr int LT = 1024;                   // threads of a listed window's block sort
constexpr int BCAP = 4096;                 // listed windows up to this size sort in shared memory
constexpr int LW = LT / 32;
static_assert(NB % 1024 == 0, "the scan kernel's 1024 threads own NB / 1024 buckets each");
static_assert(NB << BSH == 1 << 26, "the buckets cover keys below 2^26");

__device__ __forceinline__ uint32_t bucket_of(uint32_t k) {
    return min(k >> BSH, (uint32_t)(NB - 1));
}

struct TieRun {
    long long start;     // first position of the run in the sorted arrays
    long long seg_base;  // first position of its segment
    int len, pad;
};

struct BigWin {
    long long seg_base;  // first position of the segment
    int lo, n;           // the window: positions [lo, lo + n) of the segment
};

// ---------------------------------------------------------------- count / scan

// One 2,048-key sort tile per block pass: a shared-memory histogram, then one
// global atomic per non-empty bucket of the tile.
__global__ void __launch_bounds__(BT)
    k_depth_count(const uint32_t *__restrict__ keys, const SortTile *__restrict__ tiles,
                  const int *__restrict__ n_tiles_dev, uint32_t *__restrict__ count) {
    __shared__ uint32_t h[NB];
    const int tid = threadIdx.x;
    const int nt = *n_tiles_dev;
    for (int tile = blockIdx.x; tile < nt; tile += gridDim.x) {
        const SortTile T = tiles[tile];
        const uint32_t *k = keys + T.seg_base + T.t0;
        for (int d = tid; d < NB; d += BT) h[d] = 0;
        uint32_t kv[BPT];
#pragma unroll
        for (int r = 0; r < BPT; ++r) {
            const int j = r * BT + tid;
            kv[r] = j < T.nk ? k[j] : 0u;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < BPT; ++r)
            if (r * BT + tid < T.nk) atomicAdd(&h[bucket_of(kv[r])], 1u);
        __syncthreads();
        uint32_t *c = count + (long long)T.seg * NB;
        for (int d = tid; d < NB; d += BT) {
            const uint32_t v = h[d];
            if (v) atomicAdd(c + d, v);
        }
        __syncthreads();  // h is cleared for the block's next tile
    }
}

// One block of 1024 threads per camera; thread d owns buckets SPT d .. SPT d +
// SPT - 1. count becomes the scatter's cursor (the bucket's start in the
// segment); win[WPS tile_start[s] + w] = (first position, end position, first
// bucket, last bucket + 1) of window w (empty windows all zero); cut[s] = the
// segment's cut (see DepthCut): the first non-empty bucket starting at or past
// the first-phase windows' end, win1 WIN positions each.
__global__ void __launch_bounds__(1024)
    k_depth_scan(uint32_t *__restrict__ count, int4 *__restrict__ win,
                 const int *__restrict__ tile_start, DepthCut *__restrict__ cut, int prefix) {
    constexpr int SPT = NB / 1024;
    __shared__ uint32_t ws[32];
    __shared__ int wm[32];
    __shared__ int bcut;
    const int s = blockIdx.x, d = threadIdx.x, lane = d & 31, warp = d >> 5;
    if (d == 0) bcut = NB;
    uint32_t *cs = count + (long long)s * NB + SPT * d;
    uint32_t c[SPT], sum = 0;
#pragma unroll
    for (int q = 0; q < SPT; ++q) {
        c[q] = cs[q];
        sum += c[q];
    }
    const int i0 = WPS * tile_start[s], i1 = WPS * tile_start[s + 1];
    for (int i = i0 + d; i < i1; i += 1024) win[i] = make_int4(0, 0, 0, 0);
    // exclusive prefix of the counts
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) ws[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t v = ws[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += t;
        }
        ws[lane] = v;  // inclusive totals of warps 0..lane
    }
    __syncthreads();
    const int total = (int)ws[31];
    uint32_t ex[SPT];
    ex[0] = (warp ? ws[warp - 1] : 0u) + incl - sum;
#pragma unroll
    for (int q = 1; q < SPT; ++q) ex[q] = ex[q - 1] + c[q - 1];
    int m_in = -1;  // the start of this thread's last non-empty bucket
#pragma unroll
    for (int q = 0; q < SPT; ++q) {
        cs[q] = ex[q];
        if (c[q]) m_in = (int)ex[q];
    }
    // the start of the last non-empty bucket before this thread's first (-1:
    // none): exclusive max scan over the threads
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, m_in, o);
        if (lane >= o) m_in = max(m_in, v);
    }
    if (lane == 31) wm[warp] = m_in;
    int prev = __shfl_up_sync(0xffffffffu, m_in, 1);
    if (lane == 0) prev = -1;
    __syncthreads();  // win cleared, wm complete
    for (int w = 0; w < warp; ++w) prev = max(prev, wm[w]);
#pragma unroll
    for (int q = 0; q < SPT; ++q) {
        if (c[q]) {
            const int b0 = (int)ex[q], b1 = b0 + (int)c[q], w = b0 / WIN;
            const int bucket = SPT * d + q;
            if (prev < 0 || prev / WIN != w) {  // first bucket of w
                win[i0 + w].x = b0;
                win[i0 + w].z = bucket;
            }
            if (b1 == total || b1 / WIN != w) {  // last bucket of w
                win[i0 + w].y = b1;
                win[i0 + w].w = bucket + 1;
            }
            prev = b0;
        }
    }
    // the cut: the first-phase windows cover [0, T1), T1 = the prefix rounded up
    // to whole windows; the second phase starts at the first bucket (with keys)
    // whose start is at or past T1
    const int K = prefix < 0 ? total : prefix == 0 ? max(DEPTH_PREFIX_MIN, total / DEPTH_PREFIX_DIV) : prefix;
    const int win1 = (min(K, total) + WIN - 1) / WIN;
    const long long T1 = (long long)win1 * WIN;
#pragma unroll
    for (int q = 0; q < SPT; ++q)
        if (c[q] && (long long)ex[q] >= T1) {
            atomicMin(&bcut, SPT * d + q);
            break;
        }
    __syncthreads();
    const int bc = bcut;
#pragma unroll
    for (int q = 0; q < SPT; ++q)
        if (SPT * d + q == bc) cut[s] = DepthCut{(int)ex[q], bc, win1, total};
    if (bc == NB && d == 0) cut[s] = DepthCut{total, NB, win1, total};
}

// ---------------------------------------------------------------- scatter

// One sort tile per block pass: the tile grouped by bucket in shared memory
// (ranks from shared-memory atomics), the tile's share of each bucket reserved
// with one global atomic, then written out run by run (key and slot). Five
// resident blocks per SM: a block waits on its reservations' round trip, and
// more blocks hide more of it (six against four: 4.2 -> 4.0 ms per 4,096
// cameras for the whole order; with the early end of tiles without keys of the
// phase, six spilled). Phase 1: every sort tile, the keys of buckets before the
// segment's cut; phase 2: the sort tiles of the phase map, the keys of the
// cut's bucket and after.
template <int phase>
__global__ void __launch_bounds__(BT, 5)
    k_depth_scatter(const uint32_t *__restrict__ keys, uint32_t *__restrict__ dk,
                    uint32_t *__restrict__ dv, const SortTile *__restrict__ tiles,
                    const int *__restrict__ n_tiles_dev, uint32_t *__restrict__ cursor,
                    const DepthCut *__restrict__ cut, const int *__restrict__ map, int m) {
    constexpr int DPT = NB / BT;  // buckets per thread (8), read and written as uint4 pairs
    static_assert(DPT == 8, "two uint4 per thread");
    __shared__ __align__(16) uint32_t h[NB];  // counts, then where each bucket starts in the tile
    __shared__ __align__(16) int move[NB];    // segment position of the tile's bucket run minus h
    __shared__ uint32_t skey[SORT_TILE_KEYS], sval[SORT_TILE_KEYS];
    __shared__ uint32_t ws[BT / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nt = phase == 2 ? map[3] : *n_tiles_dev;
    for (int tv = blockIdx.x; tv < nt; tv += gridDim.x) {
        const int tile = phase == 2 ? phase_item(map, m, MAP_TILES, tv) : tv;
        const SortTile T = tiles[tile];
        const uint32_t bcut = (uint32_t)cut[T.seg].bucket;
        const uint32_t blo = phase == 2 ? bcut : 0u, bhi = phase == 2 ? (uint32_t)NB : bcut;
        uint32_t kv[BPT], rk[BPT];
        uint32_t in = 0;  // bit r: key r of this thread belongs to the phase
        {
            const uint32_t *k = keys + T.seg_base + T.t0;
#pragma unroll
            for (int r = 0; r < BPT; ++r) {
                const int j = r * BT + tid;
                kv[r] = j < T.nk ? k[j] : 0u;
            }
        }
#pragma unroll
        for (int r = 0; r < BPT; ++r) {
            const uint32_t b = bucket_of(kv[r]);
            in |= (r * BT + tid < T.nk && b >= blo && b < bhi) ? 1u << r : 0u;
        }
        // a tile with no key of this phase (most tiles of the first phase: its
        // keys are a camera's nearest) ends here
        if (!__syncthreads_or(in != 0u)) continue;
        for (int d = tid; d < NB; d += BT) h[d] = 0;
        __syncthreads();
#pragma unroll
        for (int r = 0; r < BPT; ++r)
            rk[r] = (in >> r) & 1u ? atomicAdd(&h[bucket_of(kv[r])], 1u) : 0u;
        __syncthreads();
        // thread tid owns buckets DPT tid .. DPT tid + DPT - 1: reserve the
        // tile's share of each, and its start within the tile (16-byte shared
        // accesses: word-wise, lanes 4 apart would share a bank)
        uint32_t c[DPT], g[DPT], sum = 0;
        uint32_t *cur = cursor + (long long)T.seg * NB;
        {
            const uint4 a = *reinterpret_cast<const uint4 *>(&h[DPT * tid]);
            const uint4 b = *reinterpret_cast<const uint4 *>(&h[DPT * tid + 4]);
            c[0] = a.x; c[1] = a.y; c[2] = a.z; c[3] = a.w;
            c[4] = b.x; c[5] = b.y; c[6] = b.z; c[7] = b.w;
        }
#pragma unroll
        for (int q = 0; q < DPT; ++q) {
            g[q] = c[q] ? atomicAdd(cur + DPT * tid + q, c[q]) : 0u;
            sum += c[q];
        }
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) ws[warp] = incl;
        __syncthreads();
        uint32_t run = incl - sum, placed = 0;  // placed: the tile's keys of this phase
        for (int w = 0; w < BT / 32; ++w) {
            run += w < warp ? ws[w] : 0u;
            placed += ws[w];
        }
        uint32_t st[DPT];
#pragma unroll
        for (int q = 0; q < DPT; ++q) {
            st[q] = run;
            run += c[q];
        }
        *reinterpret_cast<uint4 *>(&h[DPT * tid]) = make_uint4(st[0], st[1], st[2], st[3]);
        *reinterpret_cast<uint4 *>(&h[DPT * tid + 4]) = make_uint4(st[4], st[5], st[6], st[7]);
        *reinterpret_cast<int4 *>(&move[DPT * tid]) =
            make_int4((int)(g[0] - st[0]), (int)(g[1] - st[1]), (int)(g[2] - st[2]), (int)(g[3] - st[3]));
        *reinterpret_cast<int4 *>(&move[DPT * tid + 4]) =
            make_int4((int)(g[4] - st[4]), (int)(g[5] - st[5]), (int)(g[6] - st[6]), (int)(g[7] - st[7]));
        __syncthreads();
        // the tile grouped by bucket in shared memory ...
#pragma unroll
        for (int r = 0; r < BPT; ++r) {
            const int j = r * BT + tid;
            if ((in >> r) & 1u) {
                const uint32_t p = h[bucket_of(kv[r])] + rk[r];
                skey[p] = kv[r];
                sval[p] = (uint32_t)(T.t0 + j);  // the survivor's slot
            }
        }
        __syncthreads();
        // ... and written out: consecutive threads, consecutive addresses of a run
        for (int p = tid; p < (int)placed; p += BT) {
            const uint32_t key = skey[p];
            const long long at = T.seg_base + move[bucket_of(key)] + p;
            dk[at] = key;
            dv[at] = sval[p];
        }
        __syncthreads();  // shared arrays are rebuilt for the block's next tile
    }
}

// ---------------------------------------------------------------- equal keys

// A run of L <= SHORT equal keys: its slots v[0, L) put in caller-index order.
__device__ __noinline__ void order_short_run(uint32_t *v, const uint32_t *__restrict__ oidx,
                                             long long seg_base, int L) {
    uint32_t sv[SHORT], so[SHORT];
    for (int i = 0; i < L; ++i) {
        sv[i] = v[i];
        so[i] = oidx[seg_base + sv[i]];
    }
    for (int i = 1; i < L; ++i) {  // insertion by index (the indices are distinct)
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
}

__device__ __forceinline__ void list_run(TieRun *runs, long long cap, int *n_runs, long long at,
                                         long long seg_base, int L) {
    const int r = atomicAdd(n_runs, 1);
    if (r < cap) runs[r] = TieRun{at, seg_base, L, 0};
}

// ---------------------------------------------------------------- windows

__device__ __forceinline__ void list_window(BigWin *big, long long cap, int *n_big,
                                            long long seg_base, int lo, int n) {
    const int r = atomicAdd(n_big, 1);
    if (r < cap) big[r] = BigWin{seg_base, lo, n};
}

__device__ __forceinline__ void cp_async4(uint32_t *dst, const uint32_t *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(uint32_t *dst, const uint32_t *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

constexpr int SPAN = 512;  // buckets a window sorted here may span (its bounds are staged)

// One stage: a window's keys and slots, copied in 16-byte pieces from the
// 16-byte boundary at or before the window's first position (so element i of
// the window is at [shift + i], shift = first position mod 4), and its
// buckets' bounds e[j] = start of bucket bf + j (e[nb] = end of the last).
// Sizes are multiples of 4 words: every array stays 16-byte aligned.
struct WinStage {
    uint32_t k[WCAP + 8], v[WCAP + 8];
    uint32_t e[SPAN + 4];  // SPAN + 1 used
};
static_assert(sizeof(WinStage) % 16 == 0, "the bins after the stages are read as uint4");
constexpr int BW_MAX = (WPT + 3) & ~3;  // bins a thread scans: ceil(n / WT) rounded up to 4
constexpr size_t WINDOW_SMEM = 2 * sizeof(WinStage) + (size_t)WT * BW_MAX * sizeof(uint32_t);

struct WinItem {
    int4 w;          // first, end position; first bucket, last bucket + 1
    long long base;  // the segment's first position
    int seg;
};

// Item it of the phase map's windows (map == nullptr: window item it).
__device__ __forceinline__ WinItem load_item(const int4 *__restrict__ win,
                                             const SortTile *__restrict__ tiles,
                                             const int *__restrict__ map, int m, int it, int items) {
    WinItem I{make_int4(0, 0, 0, 0), 0, 0};
    if (it < items) {
        if (map) it = phase_item(map, m, MAP_WINDOWS, it);
        I.w = win[it];
        const SortTile T = tiles[it / WPS];
        I.base = T.seg_base;
        I.seg = T.seg;
    }
    return I;
}

__device__ __forceinline__ bool sorted_here(const int4 &w) {
    const int n = w.y - w.x;
    return n >= 2 && n <= WCAP && w.w - w.z <= SPAN;
}

// Starts the copies of a window (if it is sorted here) into a stage.
__device__ __forceinline__ void stage_item(const WinItem &I, const uint32_t *__restrict__ K,
                                           const uint32_t *__restrict__ V,
                                           const uint32_t *__restrict__ ends, WinStage *S) {
    if (sorted_here(I.w)) {
        const int n = I.w.y - I.w.x;
        const long long at = I.base + I.w.x;
        const long long a0 = at & ~3LL;  // the arrays are 256-byte aligned
        const int pieces = (int)((at - a0) + n + 3) >> 2;  // <= (WCAP + 6) / 4
        for (int c = threadIdx.x; c < pieces; c += WT) {
            cp_async16(S->k + 4 * c, K + a0 + 4 * c);
            cp_async16(S->v + 4 * c, V + a0 + 4 * c);
        }
        // e[j] = ends[bf + j - 1] (0 for bucket 0's start)
        const uint32_t *e = ends + (long long)I.seg * NB + I.w.z - 1;
        const int nb = I.w.w - I.w.z;
        for (int j = threadIdx.x; j <= nb; j += WT) {
            if (I.w.z + j == 0)
                S->e[0] = 0u;
            else
                cp_async4(S->e + j, e + j);
        }
    }
    cp_async_commit();
}

// A run of equal keys left for k_tie_short: its first position in the chunk
// and (segment << 6) | length (length <= BIN_MAX: equal keys share a bin).
struct EqRun {
    uint32_t pos, seg_len;
};
constexpr int LOCAL_RUNS = WT;  // runs of a window gathered before they are listed
static_assert(LOCAL_RUNS <= WT, "one thread per gathered run");

// Each block takes windows blockIdx.x, + gridDim.x, ... of the phase map;
// while it sorts one, the next is copied into the other stage. ends[seg][b]: the end of bucket b
// (the scatter's final cursor). A key of bucket b goes to one of the bucket's
// c bins by its low bits (one bin per key on average); its place is the bin's
// start plus the number of the bin's keys below it, equal keys by their staged
// position. A window's runs of equal keys are gathered in shared memory and
// listed together (one global atomic per window: a listing atomic per run,
// all on one counter, cost the pass a fifth of its time) for k_tie_short,
// which puts each in caller-index order (about one run per 100 keys on the
// full-size workloads); a run past the list's capacity is ordered by the
// window itself. Only the slots are written back: nothing after the depth
// order reads the keys.
__global__ void __launch_bounds__(WT, 4)
    k_depth_window(const uint32_t *__restrict__ K, uint32_t *__restrict__ V,
                   const uint32_t *__restrict__ oidx, const SortTile *__restrict__ tiles,
                   const int *__restrict__ map, int m, const int *__restrict__ n_tiles_dev,
                   const int4 *__restrict__ win,
                   const uint32_t *__restrict__ ends, BigWin *__restrict__ big, long long big_cap,
                   int *__restrict__ n_big, EqRun *__restrict__ eq, long long eq_cap,
                   int *__restrict__ n_eq) {
    extern __shared__ __align__(16) unsigned char wsm_raw[];
    WinStage *stages = reinterpret_cast<WinStage *>(wsm_raw);
    uint32_t *bins = reinterpret_cast<uint32_t *>(wsm_raw + 2 * sizeof(WinStage));
    __shared__ uint32_t wsum[WT / 32];
    __shared__ uint2 local_runs[LOCAL_RUNS];  // (first position in the window, length)
    __shared__ int n_local, list_base;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int items = map ? map[1] : WPS * *n_tiles_dev;
    const int G = gridDim.x;
    for (int b = tid; b < WT * BW_MAX; b += WT) bins[b] = 0;
    if (tid == 0) n_local = 0;
    int it = blockIdx.x;
    WinItem cur = load_item(win, tiles, map, m, it, items);
    stage_item(cur, K, V, ends, stages);
    WinItem nxt = load_item(win, tiles, map, m, it + G, items);
    for (int st = 0; it < items; it += G, st ^= 1) {
        cp_async_wait_all();
        __syncthreads();  // this window is staged; the other stage is free
        stage_item(nxt, K, V, ends, stages + (st ^ 1));
        const WinItem I = cur;
        cur = nxt;
        nxt = load_item(win, tiles, map, m, it + 2 * G, items);
        const int n = I.w.y - I.w.x;
        if (!sorted_here(I.w)) {
            if (n >= 2 && tid == 0) list_window(big, big_cap, n_big, I.base, I.w.x, n);
            continue;
        }
        WinStage &S = stages[st];
        const int sh = (int)((I.base + I.w.x) & 3);
        uint32_t kr[WPT], vr[WPT], br[WPT];  // key, slot, bin | rank << 16
#pragma unroll
        for (int r = 0; r < WPT; ++r) {
            if (r * WT >= n) break;
            const int i = r * WT + tid;
            if (i < n) {
                kr[r] = S.k[sh + i];
                vr[r] = S.v[sh + i];
                const uint32_t j = bucket_of(kr[r]) - (uint32_t)I.w.z;
                const uint32_t lo = S.e[j], cnt = S.e[j + 1] - lo;
                const uint32_t rel = kr[r] - ((j + (uint32_t)I.w.z) << BSH);
                const uint32_t off = j + (uint32_t)I.w.z < (uint32_t)(NB - 1)
                                         ? (rel * cnt) >> BSH
                                         : (uint32_t)(((unsigned long long)rel * cnt) >> 32);
                const uint32_t bin = lo - (uint32_t)I.w.x + off;
                br[r] = bin | (atomicAdd(&bins[bin], 1u) << 16);
            }
        }
        __syncthreads();
        // exclusive prefix over the window's n bins, BW consecutive bins per thread
        const int BW = (((n + WT - 1) / WT) + 3) & ~3;
        const int b0 = BW * tid;
        uint32_t csum = 0, cmax = 0;
        for (int q = 0; q < BW; q += 4) {
            const uint4 c = *reinterpret_cast<const uint4 *>(&bins[b0 + q]);
            csum += c.x + c.y + c.z + c.w;
            cmax = max(cmax, max(max(c.x, c.y), max(c.z, c.w)));
        }
        uint32_t incl = csum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) wsum[warp] = incl;
        if (__syncthreads_or(cmax > (uint32_t)BIN_MAX)) {
            // a crowd of (nearly) equal keys: ranking inside the bin would be slow
            if (tid == 0) list_window(big, big_cap, n_big, I.base, I.w.x, n);
            for (int q = 0; q < BW; q += 4)
                *reinterpret_cast<uint4 *>(&bins[b0 + q]) = make_uint4(0, 0, 0, 0);
            __syncthreads();  // wsum is rewritten by the next window
            continue;
        }
        uint32_t a = incl - csum;
#pragma unroll
        for (int q = 0; q < WT / 32; ++q) a += q < warp ? wsum[q] : 0u;
        {
            uint32_t run = a;
            for (int q = 0; q < BW; q += 4) {
                const uint4 c = *reinterpret_cast<const uint4 *>(&bins[b0 + q]);
                uint4 s4;
                s4.x = run;
                s4.y = s4.x + c.x;
                s4.z = s4.y + c.y;
                s4.w = s4.z + c.z;
                run = s4.w + c.w;
                *reinterpret_cast<uint4 *>(&bins[b0 + q]) = s4;
            }
        }
        __syncthreads();
        // keys grouped by bin (the slots stay in registers) ...
#pragma unroll
        for (int r = 0; r < WPT; ++r) {
            if (r * WT >= n) break;
            if (r * WT + tid < n) S.k[bins[br[r] & 0xffffu] + (br[r] >> 16)] = kr[r];
        }
        __syncthreads();
        // ... then each key's place: its bin's start, plus the bin's keys below
        // it, plus its equals staged before it; the slot goes there
#pragma unroll
        for (int r = 0; r < WPT; ++r) {
            if (r * WT >= n) break;
            if (r * WT + tid < n) {
                const uint32_t bin = br[r] & 0xffffu;
                const uint32_t first = bins[bin];
                const uint32_t end = bin + 1 < (uint32_t)n ? bins[bin + 1] : (uint32_t)n;
                const uint32_t mine = first + (br[r] >> 16);
                uint32_t less = 0, eq_before = 0, eq_all = 1;
                if (end - first > 1u) {
                    eq_all = 0;
                    for (uint32_t j = first; j < end; ++j) {
                        const uint32_t kj = S.k[j];
                        less += kj < kr[r] ? 1u : 0u;
                        eq_all += kj == kr[r] ? 1u : 0u;
                        eq_before += (kj == kr[r] && j < mine) ? 1u : 0u;
                    }
                }
                S.v[first + less + eq_before] = vr[r];
                if (eq_all > 1u && eq_before == 0u) {  // the first of a run of equal keys
                    const int l = atomicAdd(&n_local, 1);
                    if (l < LOCAL_RUNS) local_runs[l] = make_uint2(first + less, eq_all);
                }
            }
        }
        __syncthreads();
        for (int q = 0; q < BW; q += 4)
            *reinterpret_cast<uint4 *>(&bins[b0 + q]) = make_uint4(0, 0, 0, 0);
        const int nl = n_local;
        if (nl > 0) {  // the window's runs of equal keys
            if (nl > LOCAL_RUNS) {  // too many to gather: the block sort takes the window
                __syncthreads();
                if (tid == 0) {
                    n_local = 0;
                    list_window(big, big_cap, n_big, I.base, I.w.x, n);
                }
                continue;
            }
            if (tid == 0) list_base = atomicAdd(n_eq, nl);
            __syncthreads();
            if (tid < nl) {  // listed, or ordered here when past the list's end
                const uint2 R = local_runs[tid];
                const long long at = (long long)list_base + tid;
                if (at < eq_cap)
                    eq[at] = EqRun{(uint32_t)(I.base + I.w.x + R.x), ((uint32_t)I.seg << 6) | R.y};
                else
                    order_short_run(S.v + R.x, oidx, I.base, (int)R.y);
            }
            __syncthreads();
            if (tid == 0) n_local = 0;
        }
        uint32_t *ov = V + I.base + I.w.x;
        for (int i = tid; i < n; i += WT) ov[i] = S.v[i];
    }
    cp_async_wait_all();
}

// ---------------------------------------------------------------- one block, global memory

struct BlockSortSmem {
    int wcnt[LW][256 + 1];  // per warp and digit (+1: the idle lanes' digit)
    int off[256];
    uint32_t red[2][LW];
};

// Stable LSD radix sort of (ak, av)[0, L) by ak - kbase, 8 bits per pass,
// `passes` passes, by a block of LT threads; bk / bv are scratch of length L.
// The result ends in ak / av. Callers synchronise before (ak written) and
// after.
__device__ void block_sort(uint32_t *ak, uint32_t *av, uint32_t *bk, uint32_t *bv, int L,
                           uint32_t kbase, int passes, BlockSortSmem &S) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    for (int i = tid; i < LW * 257; i += LT) (&S.wcnt[0][0])[i] = 0;
    uint32_t *srcK = ak, *srcV = av, *dstK = bk, *dstV = bv;
    for (int p = 0; p < passes; ++p) {
        const int sh = 8 * p;
        if (tid < 256) S.off[tid] = 0;
        __syncthreads();
        for (int i = tid; i < L; i += LT) atomicAdd(&S.off[((srcK[i] - kbase) >> sh) & 255u], 1);
        __syncthreads();
        if (warp == 0) {  // exclusive prefix of the 256 counts, 8 per lane
            int v[8], s = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                v[q] = S.off[8 * lane + q];
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
                S.off[8 * lane + q] = run;
                run += v[q];
            }
        }
        __syncthreads();
        for (int base = 0; base < L; base += LT) {
            const int i = base + tid;
            const bool valid = i < L;
            const uint32_t key = valid ? srcK[i] : 0u, val = valid ? srcV[i] : 0u;
            const int d = valid ? (int)(((key - kbase) >> sh) & 255u) : 256;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            const int rank = __popc(peers & lt);
            if (rank == 0) S.wcnt[warp][d] = __popc(peers);
            __syncthreads();
            if (valid) {
                int pos = S.off[d] + rank;
                for (int w = 0; w < warp; ++w) pos += S.wcnt[w][d];
                dstK[pos] = key;
                dstV[pos] = val;
            }
            __syncthreads();
            if (tid < 256) {
                int s = 0;
                for (int w = 0; w < LW; ++w) {
                    s += S.wcnt[w][tid];
                    S.wcnt[w][tid] = 0;
                }
                S.off[tid] += s;
            } else if (tid < 256 + LW) {
                S.wcnt[tid - 256][256] = 0;
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
    if (srcK != ak) {
        for (int i = tid; i < L; i += LT) {
            ak[i] = srcK[i];
            av[i] = srcV[i];
        }
    }
}

// Smallest and largest of k[0, L) over the block.
__device__ __forceinline__ void block_range(const uint32_t *k, int L, BlockSortSmem &S,
                                            uint32_t &lo, uint32_t &hi) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    lo = 0xffffffffu;
    hi = 0u;
    for (int i = tid; i < L; i += LT) {
        lo = min(lo, k[i]);
        hi = max(hi, k[i]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) {
        S.red[0][warp] = lo;
        S.red[1][warp] = hi;
    }
    __syncthreads();
    for (int w = 0; w < LW; ++w) {
        lo = min(lo, S.red[0][w]);
        hi = max(hi, S.red[1][w]);
    }
    __syncthreads();  // S.red may be rewritten
}

__device__ __forceinline__ int passes_for(uint32_t span) {
    return span ? (32 - __clz(span) + 7) / 8 : 0;
}

__global__ void __launch_bounds__(LT)
    k_depth_big(uint32_t *__restrict__ K, uint32_t *__restrict__ V, uint32_t *__restrict__ SK,
                uint32_t *__restrict__ SV, const uint32_t *__restrict__ oidx,
                const BigWin *__restrict__ big, long long big_cap, const int *__restrict__ n_big,
                TieRun *__restrict__ runs, long long run_cap, int *__restrict__ n_runs) {
    __shared__ BlockSortSmem S;
    extern __shared__ __align__(16) uint32_t bsm[];  // [4][BCAP]: a window and its scratch
    const long long nb = min((long long)*n_big, big_cap);
    for (long long b = blockIdx.x; b < nb; b += gridDim.x) {
        const BigWin W = big[b];
        const long long at = W.seg_base + W.lo;
        // a window of up to BCAP keys is sorted in shared memory
        const bool local = W.n <= BCAP;
        uint32_t *ak = local ? bsm : K + at, *av = local ? bsm + BCAP : V + at;
        uint32_t *bk = local ? bsm + 2 * BCAP : SK + at, *bv = local ? bsm + 3 * BCAP : SV + at;
        if (local) {
            for (int i = threadIdx.x; i < W.n; i += LT) {
                ak[i] = K[at + i];
                av[i] = V[at + i];
            }
            __syncthreads();
        }
        uint32_t lo, hi;
        block_range(ak, W.n, S, lo, hi);
        const int passes = passes_for(hi - lo);
        if (passes) block_sort(ak, av, bk, bv, W.n, lo, passes, S);
        __syncthreads();
        for (int p = threadIdx.x; p < W.n - 1; p += LT) {
            const uint32_t kp = ak[p];
            if (ak[p + 1] == kp && (p == 0 || ak[p - 1] != kp)) {
                int e = p + 2;
                while (e < W.n && ak[e] == kp) ++e;
                if (e - p <= SHORT)
                    order_short_run(av + p, oidx, W.seg_base, e - p);
                else  // k_tie_long reads the run from K and V (written back below)
                    list_run(runs, run_cap, n_runs, at + p, W.seg_base, e - p);
            }
        }
        __syncthreads();
        if (local) {
            for (int i = threadIdx.x; i < W.n; i += LT) {
                K[at + i] = ak[i];
                V[at + i] = av[i];
            }
            __syncthreads();
        }
    }
}
constexpr size_t BIG_SMEM = 4 * BCAP * sizeof(uint32_t);

// A listed run of equal keys: the keys array holds the caller indices of its
// slots while one block sorts them, and gets the key back at the end.
__global__ void __launch_bounds__(LT)
    k_tie_long(uint32_t *__restrict__ K, uint32_t *__restrict__ V, uint32_t *__restrict__ SK,
               uint32_t *__restrict__ SV, const uint32_t *__restrict__ oidx,
               const TieRun *__restrict__ runs, long long run_cap, const int *__restrict__ n_runs) {
    __shared__ BlockSortSmem S;
    const long long nr = min((long long)*n_runs, run_cap);
    for (long long r = blockIdx.x; r < nr; r += gridDim.x) {
        const TieRun R = runs[r];
        uint32_t *ak = K + R.start, *av = V + R.start;
        const uint32_t kz = ak[0];
        __syncthreads();  // every thread has read kz before it is overwritten
        for (int i = threadIdx.x; i < R.len; i += LT) ak[i] = oidx[R.seg_base + av[i]];
        __syncthreads();
        uint32_t lo, hi;
        block_range(ak, R.len, S, lo, hi);
        block_sort(ak, av, SK + R.start, SV + R.start, R.len, 0u, passes_for(hi), S);
        __syncthreads();
        for (int i = threadIdx.x; i < R.len; i += LT) ak[i] = kz;
        __syncthreads();
    }
}

// The listed runs of equal keys (one thread per run): slots in caller-index order.
__global__ void k_tie_short(uint32_t *__restrict__ V, const uint32_t *__restrict__ oidx,
                            const long long *__restrict__ seg_start, const EqRun *__restrict__ eq,
                            long long eq_cap, const int *__restrict__ n_eq) {
    const long long ne = min((long long)*n_eq, eq_cap);
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < ne;
         r += (long long)gridDim.x * blockDim.x) {
        const EqRun R = eq[r];
        order_short_run(V + R.pos, oidx, seg_start[R.seg_len >> 6], (int)(R.seg_len & 63u));
    }
}

}  // namespace

size_t depth_window_bytes() { return sizeof(int4); }
size_t depth_big_bytes() { return sizeof(BigWin); }
size_t depth_eq_bytes() { return sizeof(EqRun); }
size_t tie_run_bytes() { return sizeof(TieRun); }

// Per device, once: SM count and resident window blocks per SM.
static cudaError_t depth_setup(int &sms, int &win_per) {
    static int sm_count[64] = {0}, win_per_sm[64] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (sm_count[dev] == 0) {
        int n_sm = 0, per = 0;
        e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_depth_window, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)WINDOW_SMEM);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_depth_big, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)BIG_SMEM);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_depth_window, WT, WINDOW_SMEM);
        if (e != cudaSuccess) return e;
        win_per_sm[dev] = std::max(per, 1);
        sm_count[dev] = n_sm;
    }
    sms = sm_count[dev];
    win_per = win_per_sm[dev];
    return cudaSuccess;
}

// The window pass and what it lists (windows for the one-block sort, runs of
// equal keys), for the windows of a phase map.
// keys / vals: the one-block sort's and the long ties' scratch.
static void depth_windows(uint32_t *keys, uint32_t *vals, uint32_t *sk, uint32_t *sv,
                          const uint32_t *oidx, const SortTile *tiles, const long long *seg_start,
                          const int *map, int m, const int *n_tiles_dev, int grid,
                          const uint32_t *ends, const int4 *w4,
                          void *big, long long big_cap, void *eq, long long eq_cap, void *runs,
                          long long run_cap, int *counters, int sms, int win_per, cudaStream_t s) {
    k_depth_window<<<std::min(WPS * grid, sms * win_per), WT, WINDOW_SMEM, s>>>(
        sk, sv, oidx, tiles, map, m, n_tiles_dev, w4, ends, (BigWin *)big, big_cap, counters + 1,
        (EqRun *)eq, eq_cap, counters + 2);
    // listed windows: keys and slots sorted through the free keys / vals arrays
    k_depth_big<<<sms, LT, BIG_SMEM, s>>>(sk, sv, keys, vals, oidx, (const BigWin *)big, big_cap,
                                          counters + 1, (TieRun *)runs, run_cap, counters);
    k_tie_long<<<sms, LT, 0, s>>>(sk, sv, keys, vals, oidx, (const TieRun *)runs, run_cap,
                                  counters);
    // last: a listed window's runs are already in order when the block sort has
    // written it, so ordering them again changes nothing
    k_tie_short<<<sms * 4, 256, 0, s>>>(sv, oidx, seg_start, (const EqRun *)eq, eq_cap,
                                        counters + 2);
}

cudaError_t launch_depth_order(uint32_t *keys, uint32_t *vals, uint32_t *sk, uint32_t *sv,
                               const uint32_t *oidx, const SortTile *tiles, const int *tile_start,
                               const long long *seg_start, int m, int grid, uint32_t *count,
                               void *win, void *big, long long big_cap, void *eq, long long eq_cap,
                               void *runs, long long run_cap, int *counters, DepthCut *cut,
                               int prefix, const int *blkpre, int bin_ranks, int *map,
                               uint32_t *scr_k, uint32_t *scr_v, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    int sms = 0, win_per = 0;
    cudaError_t e = depth_setup(sms, win_per);
    if (e != cudaSuccess) return e;
    const int *n_tiles_dev = tile_start + m;
    e = cudaMemsetAsync(count, 0, (size_t)m * NB * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(counters, 0, 3 * sizeof(int), s);
    if (e != cudaSuccess) return e;
    int4 *w4 = (int4 *)win;
    k_depth_count<<<grid, BT, 0, s>>>(keys, tiles, n_tiles_dev, count);
    k_depth_scan<<<m, 1024, 0, s>>>(count, w4, tile_start, cut, prefix);
    e = launch_phase_map(1, m, cut, nullptr, tile_start, blkpre, bin_ranks, map, nullptr, nullptr, s);
    if (e != cudaSuccess) return e;
    k_depth_scatter<1><<<grid, BT, 0, s>>>(keys, sk, sv, tiles, n_tiles_dev, count, cut, map, m);
    // the whole order (prefix < 0): every window item, no map
    depth_windows(scr_k, scr_v, sk, sv, oidx, tiles, seg_start, prefix < 0 ? nullptr : map, m,
                  n_tiles_dev, grid, count, w4, big, big_cap, eq, eq_cap, runs, run_cap, counters,
                  sms, win_per, s);
    return cudaGetLastError();
}

cudaError_t launch_depth_finish(const uint32_t *keys, uint32_t *scr_k, uint32_t *scr_v,
                                uint32_t *sk, uint32_t *sv, const uint32_t *oidx,
                                const SortTile *tiles, const long long *seg_start, int m, int grid,
                                uint32_t *count, void *win, void *big, long long big_cap, void *eq,
                                long long eq_cap, void *runs, long long run_cap, int *counters,
                                const DepthCut *cut, const int *map, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    int sms = 0, win_per = 0;
    cudaError_t e = depth_setup(sms, win_per);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(counters, 0, 3 * sizeof(int), s);
    if (e != cudaSuccess) return e;
    // (usually little or no work: a small grid, looping over the map's tiles)
    k_depth_scatter<2><<<std::min(grid, 4 * sms), BT, 0, s>>>(keys, sk, sv, tiles, nullptr, count,
                                                               cut, map, m);
    depth_windows(scr_k, scr_v, sk, sv, oidx, tiles, seg_start, map, m, nullptr, grid, count,
                  (const int4 *)win, big, big_cap, eq, eq_cap, runs, run_cap, counters, sms,
                  win_per, s);
    return cudaGetLastError();
}

}  // namespace gsk
