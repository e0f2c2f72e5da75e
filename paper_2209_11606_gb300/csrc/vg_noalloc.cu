// Counting sort into blocks that allocates no device memory.
//
// vg_insert() keeps its working buffers in the context, which grows them
// with cudaMalloc.  Some callers cannot allocate at call time: a plugin
// whose host framework owns all device memory and forbids allocation on its
// execution path, a latency-critical loop that cannot absorb the implicit
// device synchronisation of cudaMalloc/cudaFree, or a process running close
// to the memory limit where an allocation could fail half way through.
// vg_sort_blocks_noalloc() serves them: its scratch (per-particle keys and
// slots, the block counts and the scan partials) lives in one file-scope
// __device__ array of fixed size, so the call only launches kernels and
// copies a few bytes; the caller passes the positions and the two output
// arrays.  The array exists once per device that loads the library and is
// shared by every call on that device.
#include <stdio.h>
#include <string.h>

#include "vg_internal.cuh"

namespace vg {
namespace {

constexpr long long NA_MAX_N = 1ll << 20;    // particles per call
constexpr long long NA_MAX_BLK = 1ll << 18;  // blocks per call
constexpr int NA_SCAN_THREADS = 1024;
constexpr int NA_MAX_DEV = 64;

// Scratch layout (ints): key[N] | slot[N] | tmp[N] | count[BLK] | err[4]
constexpr long long NA_WORDS = 3 * NA_MAX_N + NA_MAX_BLK + 4;
static __device__ __align__(256) int na_scratch[NA_WORDS];

int *na_ptr[NA_MAX_DEV];  // device address of na_scratch, per device

__device__ __forceinline__ int na_coord(double x, double lo, double h, int n) {
    int b = (int)floor(__ddiv_rn(__dsub_rn(x, lo), h));
    return b < 0 ? 0 : (b >= n ? n - 1 : b);
}

__device__ __forceinline__ double na_wrap(double x, double lo, double L) {
    double t = __dsub_rn(x, lo);
    if (t < 0.0 || t >= L) {
        t = t - floor(t / L) * L;
        if (t >= L) t -= L;
        if (t < 0.0) t = 0.0;
    }
    return __dadd_rn(lo, t);
}

__global__ void na_clear(int *p, long long n) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) p[i] = 0;
}

// block key of each particle and its slot from an atomic capture on the count
__global__ void na_index(Grid g, long long n, const double *__restrict__ pos, int *__restrict__ key,
                         int *__restrict__ slot, int *__restrict__ count, int *__restrict__ err) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    long long k = 0, mul = 1;
    bool bad = false, outside = false;
    for (int a = 0; a < g.dim; a++) {
        double x = pos[i * g.dim + a];
        if (!isfinite(x)) { bad = true; x = g.lo[a]; }
        if (g.per[a]) x = na_wrap(x, g.lo[a], g.L[a]);
        else if (x < g.lo[a] || x > g.hi[a]) { outside = true; x = g.lo[a]; }
        k += mul * na_coord(x, g.lo[a], g.h[a], g.nb[a]);
        mul *= g.nb[a];
    }
    if (bad) atomicAdd(&err[1], 1);
    if (outside) atomicAdd(&err[0], 1);
    key[i] = (int)k;
    slot[i] = atomicAdd(&count[k], 1);
}

// exclusive scan of the block counts by one CTA (at most NA_MAX_BLK blocks)
__global__ void na_scan(const int *__restrict__ count, int *__restrict__ start, long long nblk) {
    __shared__ int part[NA_SCAN_THREADS];
    const long long per = (nblk + NA_SCAN_THREADS - 1) / NA_SCAN_THREADS;
    const long long b0 = threadIdx.x * per, b1 = min(nblk, b0 + per);
    int s = 0;
    for (long long b = b0; b < b1; b++) s += count[b];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int d = 1; d < NA_SCAN_THREADS; d <<= 1) {
        int v = threadIdx.x >= d ? part[threadIdx.x - d] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int run = part[threadIdx.x] - s;
    for (long long b = b0; b < b1; b++) {
        start[b] = run;
        run += count[b];
    }
    if (threadIdx.x == NA_SCAN_THREADS - 1) start[nblk] = part[threadIdx.x];
}

__global__ void na_scatter(long long n, const int *__restrict__ key, const int *__restrict__ slot,
                           const int *__restrict__ start, int *__restrict__ tmp) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) tmp[start[key[i]] + slot[i]] = (int)i;
}

// inside each block, order the particles by input index: a scan over a
// small block, the position in a large one (sorted in place before)
__global__ void na_order(long long n, const int *__restrict__ key, const int *__restrict__ start,
                         const int *__restrict__ tmp, int *__restrict__ order) {
    long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (u >= n) return;
    int i = tmp[u];
    int k = key[i];
    int b0 = start[k], b1 = start[k + 1], rank = 0;
    if (b1 - b0 > VG_SMALL_BLOCK) rank = (int)(u - b0);
    else
        for (int v = b0; v < b1; v++) rank += tmp[v] < i;
    order[b0 + rank] = i;
}

void set_err(char *buf, int len, const char *msg) {
    if (buf && len > 0) {
        strncpy(buf, msg, (size_t)len - 1);
        buf[len - 1] = 0;
    }
}

}  // namespace
}  // namespace vg

using namespace vg;

extern "C" vg_status vg_sort_blocks_noalloc(int dim, const double *lo, const double *hi, const int *periodic,
                                            const int *nblocks, int64_t n, const double *pos, int32_t *block_start,
                                            int32_t *order, void *stream, char *errbuf, int errlen) {
    char msg[160];
    if (dim != 2 && dim != 3) { set_err(errbuf, errlen, "dim must be 2 or 3"); return VG_ERR_ARG; }
    if (!lo || !hi || !periodic || !nblocks) { set_err(errbuf, errlen, "NULL box or grid argument"); return VG_ERR_ARG; }
    if (n < 0 || (n > 0 && (!pos || !order)) || !block_start) {
        set_err(errbuf, errlen, "bad count or NULL array");
        return VG_ERR_ARG;
    }
    if (n > NA_MAX_N) {
        snprintf(msg, sizeof msg, "%lld particles exceed the no-alloc limit of %lld", (long long)n, NA_MAX_N);
        set_err(errbuf, errlen, msg);
        return VG_ERR_ARG;
    }
    Grid g{};
    g.dim = dim;
    g.nblk = 1;
    for (int a = 0; a < 3; a++) {
        if (a < dim) {
            if (!(hi[a] > lo[a]) || nblocks[a] < 1) { set_err(errbuf, errlen, "empty box or block count < 1"); return VG_ERR_ARG; }
            g.lo[a] = lo[a]; g.hi[a] = hi[a]; g.L[a] = hi[a] - lo[a];
            g.per[a] = periodic[a] ? 1 : 0;
            g.nb[a] = nblocks[a];
        } else {
            g.lo[a] = 0; g.hi[a] = 1; g.L[a] = 1; g.per[a] = 0; g.nb[a] = 1;
        }
        g.h[a] = g.L[a] / g.nb[a];
        g.nblk *= g.nb[a];
        if (g.nblk > NA_MAX_BLK) {
            snprintf(msg, sizeof msg, "more than %lld blocks exceed the no-alloc limit", NA_MAX_BLK);
            set_err(errbuf, errlen, msg);
            return VG_ERR_ARG;
        }
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEV) {
        cudaGetLastError();
        set_err(errbuf, errlen, "no usable CUDA device");
        return VG_ERR_CUDA;
    }
    // set-up, once per device, with that device current: the host-side name
    // na_scratch is not a device address; ask the runtime for the real one
    if (!na_ptr[dev]) {
        int *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress((void **)&p, na_scratch);
        if (e != cudaSuccess || !p) {
            snprintf(msg, sizeof msg, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            set_err(errbuf, errlen, msg);
            return VG_ERR_CUDA;
        }
        na_ptr[dev] = p;
    }
    int *base = na_ptr[dev];
    int *key = base, *slot = base + NA_MAX_N, *tmp = base + 2 * NA_MAX_N;
    int *count = base + 3 * NA_MAX_N, *err = count + NA_MAX_BLK;
    cudaStream_t st = (cudaStream_t)stream;
    const int T = 256;
    // the counts and error flags must start at zero; the rest is overwritten
    na_clear<<<(unsigned)((g.nblk + T - 1) / T), T, 0, st>>>(count, g.nblk);
    na_clear<<<1, 32, 0, st>>>(err, 4);
    if (n > 0) {
        unsigned nb = (unsigned)((n + T - 1) / T);
        na_index<<<nb, T, 0, st>>>(g, n, pos, key, slot, count, err);
        na_scan<<<1, NA_SCAN_THREADS, 0, st>>>(count, block_start, g.nblk);
        na_scatter<<<nb, T, 0, st>>>(n, key, slot, block_start, tmp);
        // large blocks sorted in place: the slots serve as scratch, the block
        // counts (read by the scan already) as the list, err[2] as its length
        sort_big_blocks(block_start, g.nblk, tmp, slot, count, err + 2, 304, st);
        na_order<<<nb, T, 0, st>>>(n, key, block_start, tmp, order);
    } else {
        na_scan<<<1, NA_SCAN_THREADS, 0, st>>>(count, block_start, g.nblk);
    }
    cudaError_t e = cudaGetLastError();
    int herr[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(herr, err, sizeof herr, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        snprintf(msg, sizeof msg, "CUDA: %s", cudaGetErrorString(e));
        set_err(errbuf, errlen, msg);
        return VG_ERR_CUDA;
    }
    if (herr[1]) { set_err(errbuf, errlen, "non-finite coordinates"); return VG_ERR_NONFINITE; }
    if (herr[0]) { set_err(errbuf, errlen, "particles outside a walled box"); return VG_ERR_OUT_OF_BOX; }
    set_err(errbuf, errlen, "");
    return VG_OK;
}
