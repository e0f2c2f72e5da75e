// Counting sort of particles into the block grid, and exclusive scans.
//
// The paper's serial put() and parallel put_parallel() (Sec. 2.2.5) place a
// particle in slot co[k]++ of its block k, the latter via an atomic capture
// and an overflow buffer.  On the GPU the same atomic capture gives each
// particle a slot; an exclusive scan of the block counts then gives every
// block exact capacity, so no overflow buffer exists.  A last pass orders the
// particles inside a block by input index (the paper notes that thread timing
// otherwise changes the insertion order, Sec. 2.2.5), making the result
// deterministic.
#include "vg_internal.cuh"

namespace vg {

namespace {

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// Block coordinate of one axis: floor((x - lo)/h) clamped to [0, n-1].
__device__ __forceinline__ int block_coord(double x, double lo, double h, int n) {
    int b = (int)floor(__ddiv_rn(__dsub_rn(x, lo), h));
    return b < 0 ? 0 : (b >= n ? n - 1 : b);
}

// Wraps a periodic coordinate into [lo, hi).
__device__ __forceinline__ double wrap(double x, double lo, double L) {
    double t = __dsub_rn(x, lo);
    if (t < 0.0 || t >= L) {
        t = t - floor(t / L) * L;
        if (t >= L) t -= L;
        if (t < 0.0) t = 0.0;
    }
    return __dadd_rn(lo, t);
}

// System of input particle i: the last system whose first particle is <= i.
__device__ __forceinline__ int system_of(const Sys *sys, int nsys, long long i) {
    int lo = 0, hi = nsys - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sys[mid].p_base <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Step 1: validate, wrap, compute the global block key (the system's first
// block + the block inside the system) and take a slot with an atomic
// capture on the block count.
__global__ void k_index(const Sys *__restrict__ sys, int nsys, int dim, long long n,
                        const double *__restrict__ pos, const double *__restrict__ rad,
                        int *__restrict__ key, int *__restrict__ slot, int *__restrict__ count,
                        int *__restrict__ err) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int sidx = nsys > 1 ? system_of(sys, nsys, i) : 0;
    const Grid &g = sys[sidx].g;
    long long k = 0, mul = 1;
    bool bad = false, outside = false;
    for (int a = 0; a < dim; a++) {
        double x = pos[i * dim + a];
        if (!isfinite(x)) { bad = true; x = g.lo[a]; }
        if (g.per[a]) x = wrap(x, g.lo[a], g.L[a]);
        else if (x < g.lo[a] || x > g.hi[a]) { outside = true; x = g.lo[a]; }
        k += mul * block_coord(x, g.lo[a], g.h[a], g.nb[a]);
        mul *= g.nb[a];
    }
    if (rad && !(isfinite(rad[i]) && rad[i] >= 0.0)) bad = true;
    if (bad) atomicAdd(&err[1], 1);
    if (outside) atomicAdd(&err[0], 1);
    k += sys[sidx].blk_base;
    key[i] = (int)k;
    slot[i] = atomicAdd(&count[k], 1);
}

// Largest radius of each system (radical stop test); radii are >= 0, and
// non-negative doubles order like their bit patterns.
__global__ void k_rmax(Sys *__restrict__ sys, int nsys, long long n, const double *__restrict__ rad) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int sidx = nsys > 1 ? system_of(sys, nsys, i) : 0;
    const double r = rad[i];
    if (r > 0.0 && isfinite(r))
        atomicMax(reinterpret_cast<unsigned long long *>(&sys[sidx].rmax), (unsigned long long)__double_as_longlong(r));
}

// Step 3: scatter input indices to their (unordered) slot in the block.
__global__ void k_scatter(long long n, const int *__restrict__ key, const int *__restrict__ slot,
                          const int *__restrict__ bstart, int *__restrict__ tmp_id) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    tmp_id[bstart[key[i]] + slot[i]] = (int)i;
}

// Step 4: rank inside the block by input index and write the sorted store.
// A block of up to VG_SMALL_BLOCK particles is ranked by a scan over its
// entries; a larger one has been sorted in place by sort_big_blocks, so a
// particle's rank is its position.
__global__ void k_finalize(const Sys *__restrict__ sys, int nsys, int dim, long long n,
                           const int *__restrict__ key, const int *__restrict__ bstart,
                           const int *__restrict__ tmp_id, const double *__restrict__ pos,
                           const double *__restrict__ rad, float4 *__restrict__ p32,
                           D4 *__restrict__ p64, int *__restrict__ sid, int *__restrict__ sblk,
                           int *__restrict__ ssys) {
    long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (u >= n) return;
    const int i = tmp_id[u];
    const int k = key[i];
    const int b0 = bstart[k], b1 = bstart[k + 1];
    int rank = 0;
    if (b1 - b0 > VG_SMALL_BLOCK) rank = (int)(u - b0);
    else
        for (int v = b0; v < b1; v++) rank += tmp_id[v] < i;
    const int dst = b0 + rank;
    const int sidx = nsys > 1 ? system_of(sys, nsys, i) : 0;
    const Grid &g = sys[sidx].g;
    double x[3] = {0, 0, 0};
    float o[3] = {0.f, 0.f, 0.f};
    int kk = k - (int)sys[sidx].blk_base;
    for (int a = 0; a < dim; a++) {
        double xa = pos[(long long)i * dim + a];
        if (!isfinite(xa)) xa = g.lo[a];
        if (g.per[a]) xa = wrap(xa, g.lo[a], g.L[a]);
        else xa = fmin(fmax(xa, g.lo[a]), g.hi[a]);
        const int b = kk % g.nb[a];
        kk /= g.nb[a];
        const double corner = __dadd_rn(g.lo[a], __dmul_rn((double)b, g.h[a]));
        x[a] = xa;
        o[a] = __double2float_rn(__dsub_rn(xa, corner));
    }
    const double r = rad ? rad[i] : 0.0;
    p32[dst] = make_float4(o[0], o[1], o[2], (float)r);
    D4 v; v.x = x[0]; v.y = x[1]; v.z = x[2]; v.w = r;
    p64[dst] = v;
    sid[dst] = i;
    sblk[dst] = k;
    ssys[dst] = sidx;
}

// ---- in-place sort of the particle ids of large blocks ----------------------

constexpr int BIG_THREADS = 512;
constexpr int BIG_SMEM = 4096;  // ids sorted in shared memory up to this count
constexpr int RADIX_BITS = 4;
constexpr int RADIX = 1 << RADIX_BITS;

// The blocks that hold more than VG_SMALL_BLOCK particles.
__global__ void k_list_big(const int *__restrict__ bstart, long long nblk, int *__restrict__ list,
                           int *__restrict__ nlist) {
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k < nblk && bstart[k + 1] - bstart[k] > VG_SMALL_BLOCK) list[atomicAdd(nlist, 1)] = (int)k;
}

// Exclusive scan of RADIX * BIG_THREADS counters in shared memory (digit-major
// order), each thread scanning RADIX consecutive entries.
__device__ void cta_scan_counts(int *cnt, int *part) {
    const int t = threadIdx.x;
    int loc[RADIX], sum = 0;
#pragma unroll
    for (int d = 0; d < RADIX; d++) {
        loc[d] = sum;
        sum += cnt[t * RADIX + d];
    }
    part[t] = sum;
    __syncthreads();
    for (int off = 1; off < BIG_THREADS; off <<= 1) {
        const int v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    const int base = part[t] - sum;
#pragma unroll
    for (int d = 0; d < RADIX; d++) cnt[t * RADIX + d] = base + loc[d];
    __syncthreads();
}

// Sorts the ids of every listed block ascending, in place (a block's ids
// are distinct input indices).  Up to BIG_SMEM ids: a bitonic sort in shared
// memory.  Beyond: an LSD radix sort of (id - min) in digits of RADIX_BITS,
// each thread taking a contiguous chunk so that every pass is stable,
// ping-ponging between the block's range in `ids` and the same range in
// `scratch`.
__global__ void __launch_bounds__(BIG_THREADS) k_sort_big(const int *__restrict__ bstart, const int *__restrict__ list,
                                                         const int *__restrict__ nlist, int *__restrict__ ids,
                                                         int *__restrict__ scratch) {
    __shared__ int sm[RADIX * BIG_THREADS];  // 32 KB: bitonic keys or digit counters
    __shared__ int part[BIG_THREADS];
    __shared__ int red[2];
    const int t = threadIdx.x;
    const int nl = *nlist;
    for (int e = blockIdx.x; e < nl; e += gridDim.x) {
        const int k = list[e];
        const int b0 = bstart[k], sz = bstart[k + 1] - b0;
        if (sz <= BIG_SMEM) {
            int P = 1;
            while (P < sz) P <<= 1;
            for (int x = t; x < P; x += BIG_THREADS) sm[x] = x < sz ? ids[b0 + x] : 0x7fffffff;
            __syncthreads();
            for (int kk = 2; kk <= P; kk <<= 1) {
                for (int j = kk >> 1; j > 0; j >>= 1) {
                    for (int x = t; x < P; x += BIG_THREADS) {
                        const int y = x ^ j;
                        if (y > x) {
                            const int a = sm[x], b = sm[y];
                            if ((a > b) == ((x & kk) == 0)) { sm[x] = b; sm[y] = a; }
                        }
                    }
                    __syncthreads();
                }
            }
            for (int x = t; x < sz; x += BIG_THREADS) ids[b0 + x] = sm[x];
            __syncthreads();
            continue;
        }
        // range of the ids: the passes cover the bits of (max - min)
        if (t == 0) { red[0] = 0x7fffffff; red[1] = 0; }
        __syncthreads();
        int mn = 0x7fffffff, mx = 0;
        for (int x = t; x < sz; x += BIG_THREADS) {
            const int v = ids[b0 + x];
            mn = min(mn, v);
            mx = max(mx, v);
        }
        atomicMin(&red[0], mn);
        atomicMax(&red[1], mx);
        __syncthreads();
        mn = red[0];
        const unsigned span = (unsigned)(red[1] - mn);
        const int bits = span ? 32 - __clz(span) : 0;
        const int passes = (bits + RADIX_BITS - 1) / RADIX_BITS;
        const int chunk = (sz + BIG_THREADS - 1) / BIG_THREADS;
        const int c0 = min(sz, t * chunk), c1 = min(sz, c0 + chunk);
        int *src = ids + b0, *dst = scratch + b0;
        for (int p = 0; p < passes; p++) {
            const int shift = p * RADIX_BITS;
            int h[RADIX];
#pragma unroll
            for (int d = 0; d < RADIX; d++) h[d] = 0;
            for (int x = c0; x < c1; x++) {
                const int d = (int)(((unsigned)(src[x] - mn) >> shift) & (RADIX - 1));
#pragma unroll
                for (int dd = 0; dd < RADIX; dd++) h[dd] += d == dd;
            }
            // digit-major: counter (d, t) at d * BIG_THREADS + t, scanned in
            // that order, so equal digits keep the threads' (input) order
#pragma unroll
            for (int d = 0; d < RADIX; d++) sm[d * BIG_THREADS + t] = h[d];
            __syncthreads();
            cta_scan_counts(sm, part);
            for (int x = c0; x < c1; x++) {
                const int v = src[x];
                const int d = (int)(((unsigned)(v - mn) >> shift) & (RADIX - 1));
                dst[sm[d * BIG_THREADS + t]++] = v;
            }
            __syncthreads();
            int *tmp = src; src = dst; dst = tmp;
        }
        if (src != ids + b0)
            for (int x = t; x < sz; x += BIG_THREADS) ids[b0 + x] = src[x];
        __syncthreads();
    }
}

// ---- exclusive scan: tiles, recursive tile sums, add back ------------------

template <typename TI, typename TO>
__global__ void k_scan_tiles(const TI *__restrict__ in, TO *__restrict__ out, long long n,
                             TO *__restrict__ tile_sums) {
    __shared__ TO warp_tot[SCAN_THREADS / 32];
    long long base = blockIdx.x * (long long)SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    TO v[SCAN_ITEMS];
    TO run = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
        long long idx = base + j;
        TO x = idx < n ? (TO)in[idx] : (TO)0;
        v[j] = run;
        run += x;
    }
    // warp inclusive scan of per-thread totals
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    TO incl = run;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        TO y = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += y;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
        TO t = lane < SCAN_THREADS / 32 ? warp_tot[lane] : (TO)0;
        TO ti = t;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            TO y = __shfl_up_sync(FULL, ti, d);
            if (lane >= d) ti += y;
        }
        if (lane < SCAN_THREADS / 32) warp_tot[lane] = ti - t;  // exclusive
        if (lane == SCAN_THREADS / 32 - 1 && tile_sums) tile_sums[blockIdx.x] = ti;
    }
    __syncthreads();
    TO off = warp_tot[w] + (incl - run);
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
        long long idx = base + j;
        if (idx < n) out[idx] = v[j] + off;
    }
}

template <typename T>
__global__ void k_add_tile(T *__restrict__ out, long long n, const T *__restrict__ tile_off) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx < n) out[idx] += tile_off[idx / SCAN_TILE];
}

template <typename T>
size_t scan_tmp_bytes(long long n) {
    size_t bytes = 0;
    long long m = n;
    while (m > 1) {
        long long tiles = (m + SCAN_TILE - 1) / SCAN_TILE;
        bytes += 2 * (size_t)(tiles + 1) * sizeof(T) + 256;
        m = tiles;
        if (tiles == 1) break;
    }
    return bytes + 256;
}

// Exclusive scan of n inputs into out[0..n) (out[n] is not written here).
template <typename TI, typename TO>
cudaError_t scan_rec(const TI *in, TO *out, long long n, char *tmp, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    long long tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    TO *sums = (TO *)tmp;
    TO *sums_x = sums + (tiles + 1);
    char *next = (char *)(sums_x + (tiles + 1));
    next = (char *)(((uintptr_t)next + 255) & ~(uintptr_t)255);
    ++g_launch_count;
    k_scan_tiles<TI, TO><<<(unsigned)tiles, SCAN_THREADS, 0, st>>>(in, out, n, sums);
    if (tiles > 1) {
        cudaError_t e = scan_rec<TO, TO>(sums, sums_x, tiles, next, st);
        if (e != cudaSuccess) return e;
        ++g_launch_count;
        k_add_tile<TO><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out, n, sums_x);
    }
    return cudaGetLastError();
}

}  // namespace

size_t scan_tmp_bytes_i32(long long n) { return scan_tmp_bytes<int>(n); }
size_t scan_tmp_bytes_i64(long long n) { return scan_tmp_bytes<long long>(n); }

// out has n+1 entries: out[n] = total.
cudaError_t exclusive_scan_i32(const int *in, int *out, long long n, void *tmp, cudaStream_t st) {
    // scanning n+1 entries with the last input read as 0 yields the total
    cudaError_t e = scan_rec<int, int>(in, out, n, (char *)tmp, st);
    if (e != cudaSuccess) return e;
    return cudaSuccess;
}

cudaError_t exclusive_scan_i64_from_i32(const int *in, long long *out, long long n, void *tmp,
                                        cudaStream_t st) {
    return scan_rec<int, long long>(in, out, n, (char *)tmp, st);
}

namespace {
// total = out[n-1] + in[n-1], written to out[n]
template <typename TI, typename TO>
__global__ void k_total(const TI *in, TO *out, long long n) {
    out[n] = n > 0 ? out[n - 1] + (TO)in[n - 1] : (TO)0;
}
}  // namespace

namespace {
__global__ void k_widen(const float *__restrict__ in, double *__restrict__ out, long long n) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) out[i] = (double)in[i];
}
}  // namespace

cudaError_t widen_f32(const float *in, double *out, long long n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    ++g_launch_count;
    k_widen<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, out, n);
    return cudaGetLastError();
}

// Blocks of more than VG_SMALL_BLOCK particles get their ids sorted in place
// (ids: the scattered ids, block_start the block CSR; scratch: n ints;
// list: room for nblk ints; *nlist must be 0 on entry).
cudaError_t sort_big_blocks(const int *bstart, long long nblk, int *ids, int *scratch, int *list, int *nlist,
                            int grid, cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    ++g_launch_count;
    k_list_big<<<(unsigned)((nblk + 255) / 256), 256, 0, st>>>(bstart, nblk, list, nlist);
    ++g_launch_count;
    k_sort_big<<<grid, BIG_THREADS, 0, st>>>(bstart, list, nlist, ids, scratch);
    return cudaGetLastError();
}

cudaError_t system_rmax(Sys *sys, int nsys, long long n, const double *radii, cudaStream_t st) {
    if (n <= 0 || !radii) return cudaSuccess;
    ++g_launch_count;
    k_rmax<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(sys, nsys, n, radii);
    return cudaGetLastError();
}

cudaError_t sort_particles(const Sys *sys, int nsys, int dim, long long total_blk, long long n,
                           const double *pos, const double *radii, int *key, int *slot, int *count,
                           int *bstart, int *tmp_id, float4 *p32, D4 *p64, int *sid, int *sblk,
                           int *ssys, int *errflags, void *scan_tmp, cudaStream_t st) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(count, 0, sizeof(int) * total_blk, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(errflags, 0, sizeof(int) * 2, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(errflags + 3, 0, sizeof(int), st)) != cudaSuccess) return e;
    const int T = 256;
    const unsigned nbk = (unsigned)((n + T - 1) / T);
    if (n > 0) { ++g_launch_count; k_index<<<nbk, T, 0, st>>>(sys, nsys, dim, n, pos, radii, key, slot, count, errflags); }
    if ((e = exclusive_scan_i32(count, bstart, total_blk, scan_tmp, st)) != cudaSuccess) return e;
    ++g_launch_count;
    k_total<int, int><<<1, 1, 0, st>>>(count, bstart, total_blk);
    if (n > 0) {
        ++g_launch_count;
        k_scatter<<<nbk, T, 0, st>>>(n, key, slot, bstart, tmp_id);
        // large blocks: ids sorted in place (slots are free now; the block
        // counts, read by the scan, hold the list of large blocks)
        if ((e = sort_big_blocks(bstart, total_blk, tmp_id, slot, count, errflags + 3, 304, st)) != cudaSuccess)
            return e;
        ++g_launch_count;
        k_finalize<<<nbk, T, 0, st>>>(sys, nsys, dim, n, key, bstart, tmp_id, pos, radii, p32, p64, sid, sblk, ssys);
    }
    return cudaGetLastError();
}

// ---- cell lists -----------------------------------------------------------------

namespace {
__global__ void k_rank(const int *__restrict__ sid, long long n, int *__restrict__ rank) {
    const long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (u < n) rank[sid[u]] = (int)u;
}

__global__ void k_map(const int *__restrict__ cells, long long m, long long n, const int *__restrict__ rank,
                      int *__restrict__ out, int *__restrict__ bad) {
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= m) return;
    const int i = cells[k];
    if (i < 0 || i >= n) {
        atomicAdd(bad, 1);
        out[k] = 0;
    } else {
        out[k] = rank[i];
    }
}
}  // namespace

cudaError_t map_cells(const int *sid, long long n, const int *cells, long long m, int *rank, int *out, int *bad,
                      cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    const int T = 256;
    if (n > 0) {
        ++g_launch_count;
        k_rank<<<(unsigned)((n + T - 1) / T), T, 0, st>>>(sid, n, rank);
    }
    if (m > 0) {
        ++g_launch_count;
        k_map<<<(unsigned)((m + T - 1) / T), T, 0, st>>>(cells, m, n, rank, out, bad);
    }
    return cudaGetLastError();
}

// ---- CSR compaction of faces ---------------------------------------------------

namespace {
// Faces of cell i that the CSR takes: none unless the cell is complete and
// its faces fit in the bump buffer (after an overflow the cell kernel skips
// the write, so its slots hold nothing to copy).
__global__ void k_nf_ok(long long n, const int *nf, const unsigned char *status, const long long *fptr,
                        long long fcap, int *nf_ok) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bool ok = status[i] == VG_CELL_OK && fptr[i] >= 0 && fptr[i] + nf[i] <= fcap;
    nf_ok[i] = ok ? nf[i] : 0;
}

// One warp per 32 consecutive cells: their faces are contiguous in the CSR
// ([face_off[c0], face_off[c0 + 32])), so the warp walks that output range 32
// faces at a time with coalesced stores.  In each window of 32 outputs every
// lane (one per cell) marks in shared memory the outputs its cell owns; each
// lane then copies the one face it writes.
constexpr int COMPACT_THREADS = 256;
__global__ void __launch_bounds__(COMPACT_THREADS) k_compact(long long n, const int *__restrict__ nf_ok,
                                                            const long long *__restrict__ fptr,
                                                            const int2 *__restrict__ faces,
                                                            const long long *__restrict__ face_off,
                                                            int *__restrict__ nbr_id, signed char *__restrict__ nbr_img,
                                                            unsigned char *__restrict__ face_order) {
    __shared__ unsigned char owner[COMPACT_THREADS / 32][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const long long c0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) - lane;
    if (c0 >= n) return;  // whole warps leave together
    const long long c = c0 + lane;
    const bool in = c < n;
    const long long off = in ? face_off[c] : face_off[n];
    const int cnt = in ? nf_ok[c] : 0;
    const long long src = in ? fptr[c] : 0;
    const long long base = __shfl_sync(FULL, off, 0);
    const long long end = __shfl_sync(FULL, off + cnt, 31);
    for (long long w0 = base; w0 < end; w0 += 32) {
        // this lane's cell covers outputs [off, off + cnt) of the window [w0, w0 + 32)
        const long long a = off > w0 ? off : w0, b = off + cnt < w0 + 32 ? off + cnt : w0 + 32;
        for (long long f = a; f < b; f++) owner[wib][f - w0] = (unsigned char)lane;
        __syncwarp();
        const long long f = w0 + lane;
        const int o = f < end ? (int)owner[wib][lane] : 0;
        const long long s_o = __shfl_sync(FULL, src, o);
        const long long off_o = __shfl_sync(FULL, off, o);
        if (f < end) {
            const int2 e = faces[s_o + (f - off_o)];
            nbr_id[f] = e.x;
            nbr_img[f * 3 + 0] = (signed char)(e.y & 0xff);
            nbr_img[f * 3 + 1] = (signed char)((e.y >> 8) & 0xff);
            nbr_img[f * 3 + 2] = (signed char)((e.y >> 16) & 0xff);
            face_order[f] = (unsigned char)((unsigned)e.y >> 24);
        }
        __syncwarp();
    }
}

}  // namespace

cudaError_t compact_faces(long long n, const int *nf, const unsigned char *status,
                          const long long *fptr, const int2 *faces, long long fcap, long long *face_off,
                          int *nbr_id, signed char *nbr_img, unsigned char *face_order,
                          void *scan_tmp, cudaStream_t st) {
    // scan_tmp holds n ints for the per-cell face counts, then the scan's own
    // scratch (the caller sizes it for both)
    int *nf_ok = (int *)scan_tmp;
    char *tmp = (char *)scan_tmp + (((size_t)n * sizeof(int) + 255) & ~(size_t)255);
    const int T = 256;
    unsigned nbk = (unsigned)((n + T - 1) / T);
    if (n > 0) { ++g_launch_count; k_nf_ok<<<nbk, T, 0, st>>>(n, nf, status, fptr, fcap, nf_ok); }
    cudaError_t e = scan_rec<int, long long>(nf_ok, face_off, n, tmp, st);
    if (e != cudaSuccess) return e;
    ++g_launch_count;
    k_total<int, long long><<<1, 1, 0, st>>>(nf_ok, face_off, n);
    if (n > 0) {
        ++g_launch_count;
        k_compact<<<(unsigned)((n + COMPACT_THREADS - 1) / COMPACT_THREADS), COMPACT_THREADS, 0, st>>>(
            n, nf_ok, fptr, faces, face_off, nbr_id, nbr_img, face_order);
    }
    return cudaGetLastError();
}

}  // namespace vg
