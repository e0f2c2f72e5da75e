// The learned candidate-count predictor: features, labels, training and
// inference kernels.
//
// The paper's cells take their candidates from the block walk with the
// radius bound (Sec. 2.1.3).  The prefetch form of the cell kernel instead
// preloads, in one batch, the candidates inside a ball that should hold k of
// them, sorts them by distance and cuts them in order; the radius bound still
// decides, and a shortfall falls back to the walk, so the cells do not depend
// on k.  This file predicts k per block from the particle counts of the 27
// surrounding blocks with a small network (27 -> 32 -> 32 -> 1, ReLU, FP16
// weights, FP32 accumulation), trained on the counts a finished computation
// provides: k*_i, the number of candidates within 2 R_i of cell i.
//
// Parameters are packed as W1 (32 x 27, row per hidden unit), b1, W2 (32 x
// 32), b2, W3 (32), b3: 1985 floats.  Training keeps FP32 master weights and
// Adam moments and refreshes the FP16 copy that the forward pass and the
// inference kernel read, so training sees the network that inference runs.
#include <cuda_fp16.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "vg_internal.cuh"

namespace vg {
namespace {

constexpr int NIN = 27, H1 = 32, H2 = 32;
constexpr int OW1 = 0;
constexpr int OB1 = OW1 + H1 * NIN;  // 864
constexpr int OW2 = OB1 + H1;        // 896
constexpr int OB2 = OW2 + H2 * H1;   // 1920
constexpr int OW3 = OB2 + H2;        // 1952
constexpr int OB3 = OW3 + H2;        // 1984
constexpr int NP = OB3 + 1;          // 1985
constexpr int NPS = NP + 1;          // a CTA's partial sums: gradient, then its loss sum
constexpr int SW = 1988;             // smem floats for the weights (padded)
constexpr int TS = 128;              // samples per CTA in training

// What the forward pass reads: FP16 weights, FP32 biases.
struct MlpInf {
    __half w1[H1 * NIN];
    __half w2[H2 * H1];
    __half w3[H2];
    float b1[H1], b2[H2], b3;
};

__device__ __forceinline__ int fdiv(int a, int b) {
    int q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) q--;
    return q;
}

// Packed parameters in shared memory as floats (weights widened from FP16).
__device__ void load_weights(const MlpInf *__restrict__ W, float *sw) {
    for (int u = threadIdx.x; u < NP; u += blockDim.x) {
        float v;
        if (u < OB1) v = __half2float(W->w1[u]);
        else if (u < OW2) v = W->b1[u - OB1];
        else if (u < OB2) v = __half2float(W->w2[u - OW2]);
        else if (u < OW3) v = W->b2[u - OB2];
        else if (u < OB3) v = __half2float(W->w3[u - OW3]);
        else v = W->b3;
        sw[u] = v;
    }
}

// y = W3 . relu(W2 relu(W1 x + b1) + b2) + b3, FP32 accumulation.
__device__ __forceinline__ float forward(const float *sw, const float *x, float *z1, float *z2) {
#pragma unroll 4
    for (int i = 0; i < H1; i++) {
        float a = sw[OB1 + i];
#pragma unroll
        for (int j = 0; j < NIN; j++) a = fmaf(sw[OW1 + i * NIN + j], x[j], a);
        z1[i] = a;
    }
    float y = sw[OB3];
#pragma unroll 4
    for (int k = 0; k < H2; k++) {
        float a = sw[OB2 + k];
#pragma unroll
        for (int i = 0; i < H1; i++) a = fmaf(sw[OW2 + k * H1 + i], fmaxf(z1[i], 0.f), a);
        z2[k] = a;
        y = fmaf(sw[OW3 + k], fmaxf(a, 0.f), y);
    }
    return y;
}

// System of global block b: the last system whose first block is <= b.
__device__ __forceinline__ int system_of_block(const Sys *sys, int nsys, long long b) {
    int lo = 0, hi = nsys - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sys[mid].blk_base <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// The 27 features of global block b: the counts c_j of the blocks
// b + (dx, dy, dz), index (dx+1) + 3 (dy+1) + 9 (dz+1), wrapped on periodic
// axes and 0 outside a wall, over their mean m = (sum c_j) / (blocks inside
// the box), minus 1 (0 everywhere when m = 0): the same at any density or
// block size.
__device__ void block_features(const Sys *sys, int nsys, const int *__restrict__ bstart, long long b, float *x) {
    const Sys &sy = sys[nsys > 1 ? system_of_block(sys, nsys, b) : 0];
    const Grid &g = sy.g;
    const long long kl = b - sy.blk_base;
    const int c0 = (int)(kl % g.nb[0]), c1 = (int)((kl / g.nb[0]) % g.nb[1]), c2 = (int)(kl / ((long long)g.nb[0] * g.nb[1]));
    int sum = 0, inside = 0;
    for (int j = 0; j < NIN; j++) {
        int t[3] = {c0 + j % 3 - 1, c1 + (j / 3) % 3 - 1, c2 + j / 9 - 1};
        bool ok = true;
        for (int a = 0; a < 3; a++) {
            if (t[a] >= 0 && t[a] < g.nb[a]) continue;
            if (g.per[a]) t[a] -= fdiv(t[a], g.nb[a]) * g.nb[a];
            else ok = false;
        }
        int cnt = 0;
        if (ok) {
            const long long k = sy.blk_base + t[0] + (long long)g.nb[0] * (t[1] + (long long)g.nb[1] * t[2]);
            cnt = bstart[k + 1] - bstart[k];
            inside++;
        }
        sum += cnt;
        x[j] = (float)cnt;
    }
    // x_j = c_j / m - 1 = c_j * inside / sum - 1, the quotient correctly rounded
    const float f = sum > 0 ? __fdiv_rn((float)inside, (float)sum) : 0.f;
    for (int j = 0; j < NIN; j++) x[j] = sum > 0 ? __fsub_rn(__fmul_rn(x[j], f), 1.f) : 0.f;
}

__global__ void k_features(const Sys *sys, int nsys, const int *__restrict__ bstart, long long nblk,
                           float *__restrict__ X) {
    const long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (b >= nblk) return;
    float x[NIN];
    block_features(sys, nsys, bstart, b, x);
    for (int j = 0; j < NIN; j++) X[b * NIN + j] = x[j];
}

// k*_i: candidates (particle, image) within 2 R_i of particle i, the particle
// itself excluded; one warp per cell, lanes over the blocks within reach.
__global__ void k_kstar(const Sys *sys, const D4 *__restrict__ p64, const int *__restrict__ sid,
                        const int *__restrict__ sblk, const int *__restrict__ ssys, const int *__restrict__ bstart,
                        const float *__restrict__ rfin, int nsys, long long n, int *__restrict__ kstar) {
    const int lane = threadIdx.x & 31;
    const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long u = w0; u < n; u += nw) {
        const int i = sid[u];
        const double R = (double)rfin[i];
        if (!(R > 0.0)) {
            if (lane == 0) kstar[i] = 0;
            continue;
        }
        const Sys &sy = sys[nsys > 1 ? ssys[u] : 0];
        const Grid &g = sy.g;
        const long long kl = sblk[u] - sy.blk_base;
        const int b[3] = {(int)(kl % g.nb[0]), (int)((kl / g.nb[0]) % g.nb[1]),
                          (int)(kl / ((long long)g.nb[0] * g.nb[1]))};
        const D4 p = p64[u];
        const double pp[3] = {p.x, p.y, p.z};
        const double R2 = 4.0 * R * R;
        int reach[3];
        for (int a = 0; a < 3; a++) reach[a] = a < g.dim ? (int)ceil(2.0 * R / g.h[a]) : 0;
        const long long w[3] = {2 * reach[0] + 1, 2 * reach[1] + 1, 2 * reach[2] + 1};
        const long long total = w[0] * w[1] * w[2];
        int cnt = 0;
        for (long long o = lane; o < total; o += 32) {
            const int off[3] = {(int)(o % w[0]) - reach[0], (int)((o / w[0]) % w[1]) - reach[1],
                                (int)(o / (w[0] * w[1])) - reach[2]};
            int t[3], m[3];
            bool ok = true;
            double lb2 = 0.0;
            for (int a = 0; a < 3; a++) {
                t[a] = b[a] + off[a];
                m[a] = 0;
                if (t[a] < 0 || t[a] >= g.nb[a]) {
                    if (!g.per[a]) { ok = false; break; }
                    m[a] = fdiv(t[a], g.nb[a]);
                    t[a] -= m[a] * g.nb[a];
                }
                // distance from the particle to the block's box, this axis
                const double lo = g.lo[a] + (t[a] + (double)m[a] * g.nb[a]) * g.h[a];
                const double hi = lo + g.h[a];
                const double d = pp[a] < lo ? lo - pp[a] : (pp[a] > hi ? pp[a] - hi : 0.0);
                lb2 += d * d;
            }
            if (!ok || lb2 >= R2) continue;
            const long long k = sy.blk_base + t[0] + (long long)g.nb[0] * (t[1] + (long long)g.nb[1] * t[2]);
            const bool home = m[0] == 0 && m[1] == 0 && m[2] == 0;
            for (int v = bstart[k]; v < bstart[k + 1]; v++) {
                const D4 q = p64[v];
                const double qx = q.x + m[0] * g.L[0] - pp[0];
                const double qy = q.y + m[1] * g.L[1] - pp[1];
                const double qz = q.z + m[2] * g.L[2] - pp[2];
                if (qx * qx + qy * qy + qz * qz < R2 && !(home && v == u)) cnt++;
            }
        }
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) cnt += __shfl_xor_sync(FULL, cnt, s);
        if (lane == 0) kstar[i] = cnt;
    }
}

// Largest k* of each block (-1: no particle).
__global__ void k_block_max(const int *__restrict__ sid, const int *__restrict__ sblk, const int *__restrict__ kstar,
                            long long n, int *__restrict__ kmax) {
    const long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (u < n) atomicMax(&kmax[sblk[u]], kstar[sid[u]]);
}

__global__ void k_fill(int *p, long long n, int v) {
    const long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (u < n) p[u] = v;
}

__global__ void k_flags(const int *__restrict__ kmax, long long n, int *__restrict__ flag) {
    const long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (u < n) flag[u] = kmax[u] >= 0 ? 1 : 0;
}

// Rows of blocks holding a particle, in block order: features and target
// t = log(max(1, k*max)).
__global__ void k_gather_rows(const float *__restrict__ F, const int *__restrict__ kmax,
                              const int *__restrict__ pos, long long n, float *__restrict__ X,
                              float *__restrict__ t) {
    const long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (b >= n || kmax[b] < 0) return;
    const long long r = pos[b];
    for (int j = 0; j < NIN; j++) X[r * NIN + j] = F[b * NIN + j];
    t[r] = logf((float)max(1, kmax[b]));
}

// Forward and backward pass over TS samples per CTA.  The CTA's sums of the
// gradient over its samples, and of its loss terms, go to its own row of
// `partial` (reduced afterwards in a fixed order, so the result does not
// depend on scheduling).
__global__ void __launch_bounds__(TS) k_fwdbwd(const MlpInf *__restrict__ W, const float *__restrict__ X,
                                               const float *__restrict__ t, long long M, float u, float invM,
                                               float *__restrict__ partial) {
    extern __shared__ float sm[];
    float *sw = sm;
    float *sx = sw + SW;            // TS x 27 inputs
    float *sh1 = sx + TS * NIN;     // TS x 32 relu(z1)
    float *sh2 = sh1 + TS * H1;     // TS x 32 relu(z2)
    float *sg1 = sh2 + TS * H2;     // TS x 32 dL/dz1
    float *sg2 = sg1 + TS * H1;     // TS x 32 dL/dz2
    float *sgy = sg2 + TS * H2;     // TS dL/dy
    float *sl = sgy + TS;           // TS loss terms
    load_weights(W, sw);
    const int tid = threadIdx.x;
    const long long r0 = blockIdx.x * (long long)TS;
    const long long rows = min((long long)TS, M - r0);
    for (long long q = tid; q < TS * NIN; q += TS) sx[q] = q < rows * NIN ? X[r0 * NIN + q] : 0.f;
    __syncthreads();
    float z1[H1], z2[H2];
    const float y = forward(sw, sx + tid * NIN, z1, z2);
    const bool valid = tid < rows;
    float gy = 0.f, lt = 0.f;
    if (valid) {
        const float e = y - t[r0 + tid];
        const float wgt = e < 0.f ? u : 1.f;
        gy = 2.f * wgt * e * invM;
        lt = wgt * e * e;
    }
    float g2[H2];
#pragma unroll
    for (int k = 0; k < H2; k++) {
        g2[k] = z2[k] > 0.f ? gy * sw[OW3 + k] : 0.f;
        sh2[tid * H2 + k] = fmaxf(z2[k], 0.f);
        sg2[tid * H2 + k] = g2[k];
    }
#pragma unroll 4
    for (int i = 0; i < H1; i++) {
        float a = 0.f;
#pragma unroll
        for (int k = 0; k < H2; k++) a = fmaf(g2[k], sw[OW2 + k * H1 + i], a);
        sg1[tid * H1 + i] = z1[i] > 0.f ? a : 0.f;
        sh1[tid * H1 + i] = fmaxf(z1[i], 0.f);
    }
    sgy[tid] = gy;
    sl[tid] = lt;
    __syncthreads();
    float *out = partial + blockIdx.x * (long long)NPS;
    for (int p = tid; p < NPS; p += TS) {
        float acc = 0.f;
        if (p < OB1) {
            const int i = p / NIN, j = p % NIN;
            for (int s = 0; s < TS; s++) acc = fmaf(sg1[s * H1 + i], sx[s * NIN + j], acc);
        } else if (p < OW2) {
            for (int s = 0; s < TS; s++) acc += sg1[s * H1 + (p - OB1)];
        } else if (p < OB2) {
            const int k = (p - OW2) / H1, i = (p - OW2) % H1;
            for (int s = 0; s < TS; s++) acc = fmaf(sg2[s * H2 + k], sh1[s * H1 + i], acc);
        } else if (p < OW3) {
            for (int s = 0; s < TS; s++) acc += sg2[s * H2 + (p - OB2)];
        } else if (p < OB3) {
            for (int s = 0; s < TS; s++) acc = fmaf(sgy[s], sh2[s * H2 + (p - OW3)], acc);
        } else if (p == OB3) {
            for (int s = 0; s < TS; s++) acc += sgy[s];
        } else {
            for (int s = 0; s < TS; s++) acc += sl[s];
        }
        out[p] = acc;
    }
}

// Sum of the CTAs' partial rows, in CTA order: gradient and loss sum.
__global__ void k_reduce(const float *__restrict__ partial, int nblk, float *__restrict__ grad) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NPS) return;
    float acc = 0.f;
    for (int c = 0; c < nblk; c++) acc += partial[(long long)c * NPS + p];
    grad[p] = acc;
}

// Adam on the FP32 master weights, then the FP16 copy.
__global__ void k_adam(float *__restrict__ master, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ grad, float lr, float c1, float c2, MlpInf *__restrict__ W) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NP) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float g = grad[p];
    const float mm = b1 * m[p] + (1.f - b1) * g;
    const float vv = b2 * v[p] + (1.f - b2) * g * g;
    m[p] = mm;
    v[p] = vv;
    const float w = master[p] - lr * (mm * c1) / (sqrtf(vv * c2) + eps);
    master[p] = w;
    if (p < OB1) W->w1[p] = __float2half_rn(w);
    else if (p < OW2) W->b1[p - OB1] = w;
    else if (p < OB2) W->w2[p - OW2] = __float2half_rn(w);
    else if (p < OW3) W->b2[p - OB2] = w;
    else if (p < OB3) W->w3[p - OW3] = __float2half_rn(w);
    else W->b3 = w;
}

// FP16 copy from the master weights.
__global__ void k_refresh(const float *__restrict__ master, MlpInf *__restrict__ W) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NP) return;
    const float w = master[p];
    if (p < OB1) W->w1[p] = __float2half_rn(w);
    else if (p < OW2) W->b1[p - OB1] = w;
    else if (p < OB2) W->w2[p - OW2] = __float2half_rn(w);
    else if (p < OW3) W->b2[p - OB2] = w;
    else if (p < OB3) W->w3[p - OW3] = __float2half_rn(w);
    else W->b3 = w;
}

__global__ void k_infer(const MlpInf *__restrict__ W, const float *__restrict__ X, long long M, float *__restrict__ y) {
    __shared__ float sw[SW];
    load_weights(W, sw);
    __syncthreads();
    const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (r >= M) return;
    float x[NIN], z1[H1], z2[H2];
    for (int j = 0; j < NIN; j++) x[j] = X[r * NIN + j];
    y[r] = forward(sw, x, z1, z2);
}

// Per-block preload target for the cell kernel: clamp(alpha exp(y), kmin, kmax).
__global__ void k_predict(const MlpInf *__restrict__ W, const Sys *sys, int nsys, const int *__restrict__ bstart,
                          long long nblk, float alpha, float kmin, float kmax, float *__restrict__ kblock) {
    __shared__ float sw[SW];
    load_weights(W, sw);
    __syncthreads();
    const long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (b >= nblk) return;
    float x[NIN], z1[H1], z2[H2];
    block_features(sys, nsys, bstart, b, x);
    const float y = forward(sw, x, z1, z2);
    kblock[b] = fminf(fmaxf(alpha * expf(fminf(y, 20.f)), kmin), kmax);
}

unsigned nblocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_predict(const void *weights, const Sys *sys, int nsys, const int *bstart, long long nblk,
                           float alpha, float kmin, float kmax, float *kblock, cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    ++g_launch_count;
    k_predict<<<nblocks_for(nblk, 128), 128, 0, st>>>((const MlpInf *)weights, sys, nsys, bstart, nblk, alpha, kmin,
                                                      kmax, kblock);
    return cudaGetLastError();
}

const void *mlp_weights(const vg_mlp *m);

}  // namespace vg

using namespace vg;

struct vg_mlp {
    cudaStream_t stream = nullptr;
    float *d_master = nullptr, *d_m = nullptr, *d_v = nullptr, *d_grad = nullptr;
    float *d_partial = nullptr;
    long long partial_rows = 0;
    MlpInf *d_inf = nullptr;
    long long step = 0;
    std::string err;
};

const void *vg::mlp_weights(const vg_mlp *m) { return m ? (const void *)m->d_inf : nullptr; }

namespace {

vg_status mfail(vg_mlp *m, vg_status s, const std::string &msg) {
    if (m) m->err = msg;
    return s;
}

vg_status mcuda(vg_mlp *m, cudaError_t e, const char *where) {
    return mfail(m, e == cudaErrorMemoryAllocation ? VG_ERR_OOM : VG_ERR_CUDA,
                 std::string(where) + ": " + cudaGetErrorString(e));
}

vg_status cfail(vg_ctx *c, vg_status s, const std::string &msg) {
    if (c) c->err = msg;
    return s;
}

vg_status ccuda(vg_ctx *c, cudaError_t e, const char *where) {
    return cfail(c, e == cudaErrorMemoryAllocation ? VG_ERR_OOM : VG_ERR_CUDA,
                 std::string(where) + ": " + cudaGetErrorString(e));
}

#define M_CUDA(call)                                         \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return mcuda(m, e_, #call);   \
    } while (0)
#define C_CUDA(call)                                         \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return ccuda(c, e_, #call);   \
    } while (0)

template <typename T>
cudaError_t grow(T *&p, long long &cap, long long need) {
    if (p && need <= cap) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc((void **)&p, sizeof(T) * (size_t)std::max<long long>(need, 1));
    if (e == cudaSuccess) cap = need;
    return e;
}

constexpr size_t FWD_SMEM = sizeof(float) * (SW + TS * NIN + 4 * TS * 32 + 2 * TS);

// Forward + backward over M rows and the fixed-order reduction into d_grad
// (gradient, then the loss sum in d_grad[NP]).
vg_status run_grad(vg_mlp *m, const float *X, const float *t, long long M, float u) {
    const long long nb = (M + TS - 1) / TS;
    M_CUDA(grow(m->d_partial, m->partial_rows, nb * NPS));
    ++g_launch_count;
    k_fwdbwd<<<(unsigned)nb, TS, FWD_SMEM, m->stream>>>(m->d_inf, X, t, M, u, 1.f / (float)M, m->d_partial);
    M_CUDA(cudaGetLastError());
    ++g_launch_count;
    k_reduce<<<nblocks_for(NPS, 256), 256, 0, m->stream>>>(m->d_partial, (int)nb, m->d_grad);
    M_CUDA(cudaGetLastError());
    return VG_OK;
}

}  // namespace

extern "C" {

vg_status vg_mlp_create(vg_mlp **out, void *stream) {
    if (!out) return VG_ERR_ARG;
    *out = nullptr;
    vg_mlp *m = new (std::nothrow) vg_mlp();
    if (!m) return VG_ERR_OOM;
    m->stream = (cudaStream_t)stream;
    cudaError_t e = cudaMalloc((void **)&m->d_master, sizeof(float) * NP);
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->d_m, sizeof(float) * NP);
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->d_v, sizeof(float) * NP);
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->d_grad, sizeof(float) * NPS);
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->d_inf, sizeof(MlpInf));
    if (e == cudaSuccess) e = cudaMemsetAsync(m->d_master, 0, sizeof(float) * NP, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->d_m, 0, sizeof(float) * NP, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->d_v, 0, sizeof(float) * NP, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->d_inf, 0, sizeof(MlpInf), m->stream);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fwdbwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)FWD_SMEM);
    if (e != cudaSuccess) {
        cudaGetLastError();
        vg_mlp_destroy(m);
        return e == cudaErrorMemoryAllocation ? VG_ERR_OOM : VG_ERR_CUDA;
    }
    *out = m;
    return VG_OK;
}

void vg_mlp_destroy(vg_mlp *m) {
    if (!m) return;
    if (m->d_master) cudaFree(m->d_master);
    if (m->d_m) cudaFree(m->d_m);
    if (m->d_v) cudaFree(m->d_v);
    if (m->d_grad) cudaFree(m->d_grad);
    if (m->d_partial) cudaFree(m->d_partial);
    if (m->d_inf) cudaFree(m->d_inf);
    delete m;
}

const char *vg_mlp_last_error(vg_mlp *m) { return m ? m->err.c_str() : "null predictor"; }

vg_status vg_mlp_set_params(vg_mlp *m, const float *params) {
    if (!m) return VG_ERR_ARG;
    if (!params) return mfail(m, VG_ERR_ARG, "params is NULL");
    M_CUDA(cudaMemcpyAsync(m->d_master, params, sizeof(float) * NP, cudaMemcpyHostToDevice, m->stream));
    M_CUDA(cudaMemsetAsync(m->d_m, 0, sizeof(float) * NP, m->stream));
    M_CUDA(cudaMemsetAsync(m->d_v, 0, sizeof(float) * NP, m->stream));
    ++g_launch_count;
    k_refresh<<<nblocks_for(NP, 256), 256, 0, m->stream>>>(m->d_master, m->d_inf);
    M_CUDA(cudaGetLastError());
    M_CUDA(cudaStreamSynchronize(m->stream));
    m->step = 0;
    return VG_OK;
}

vg_status vg_mlp_get_params(vg_mlp *m, float *params) {
    if (!m) return VG_ERR_ARG;
    if (!params) return mfail(m, VG_ERR_ARG, "params is NULL");
    M_CUDA(cudaMemcpyAsync(params, m->d_master, sizeof(float) * NP, cudaMemcpyDeviceToHost, m->stream));
    M_CUDA(cudaStreamSynchronize(m->stream));
    return VG_OK;
}

vg_status vg_mlp_loss_grad(vg_mlp *m, const float *X, const float *t, int64_t M, float u, double *loss,
                           float *grad) {
    if (!m) return VG_ERR_ARG;
    if (M < 1 || !X || !t) return mfail(m, VG_ERR_ARG, "empty or NULL training rows");
    vg_status s = run_grad(m, X, t, M, u);
    if (s != VG_OK) return s;
    std::vector<float> h(NPS);
    M_CUDA(cudaMemcpyAsync(h.data(), m->d_grad, sizeof(float) * NPS, cudaMemcpyDeviceToHost, m->stream));
    M_CUDA(cudaStreamSynchronize(m->stream));
    if (grad) memcpy(grad, h.data(), sizeof(float) * NP);
    if (loss) *loss = (double)h[NP] / (double)M;
    return VG_OK;
}

vg_status vg_mlp_train(vg_mlp *m, const float *X, const float *t, int64_t M, float u, float lr, int steps,
                       float *losses) {
    if (!m) return VG_ERR_ARG;
    if (M < 1 || !X || !t || steps < 0) return mfail(m, VG_ERR_ARG, "empty or NULL training rows");
    if (!(lr > 0.f)) return mfail(m, VG_ERR_ARG, "learning rate");
    float *d_loss = nullptr;
    if (losses && steps > 0) M_CUDA(cudaMalloc((void **)&d_loss, sizeof(float) * steps));
    for (int k = 0; k < steps; k++) {
        vg_status s = run_grad(m, X, t, M, u);
        if (s != VG_OK) { if (d_loss) cudaFree(d_loss); return s; }
        if (d_loss) {
            cudaError_t e = cudaMemcpyAsync(d_loss + k, m->d_grad + NP, sizeof(float), cudaMemcpyDeviceToDevice,
                                            m->stream);
            if (e != cudaSuccess) { cudaFree(d_loss); return mcuda(m, e, "loss copy"); }
        }
        m->step++;
        const double c1 = 1.0 / (1.0 - pow(0.9, (double)m->step));
        const double c2 = 1.0 / (1.0 - pow(0.999, (double)m->step));
        ++g_launch_count;
        k_adam<<<nblocks_for(NP, 256), 256, 0, m->stream>>>(m->d_master, m->d_m, m->d_v, m->d_grad, lr, (float)c1,
                                                              (float)c2, m->d_inf);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) { if (d_loss) cudaFree(d_loss); return mcuda(m, e, "k_adam"); }
    }
    if (d_loss) {
        std::vector<float> h(steps);
        cudaError_t e = cudaMemcpyAsync(h.data(), d_loss, sizeof(float) * steps, cudaMemcpyDeviceToHost, m->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
        cudaFree(d_loss);
        if (e != cudaSuccess) return mcuda(m, e, "loss readback");
        for (int k = 0; k < steps; k++) losses[k] = h[k] / (float)M;
    } else {
        M_CUDA(cudaStreamSynchronize(m->stream));
    }
    return VG_OK;
}

vg_status vg_mlp_infer(vg_mlp *m, const float *X, int64_t M, float *y) {
    if (!m) return VG_ERR_ARG;
    if (M < 0 || (M > 0 && (!X || !y))) return mfail(m, VG_ERR_ARG, "bad rows");
    if (M == 0) return VG_OK;
    ++g_launch_count;
    k_infer<<<nblocks_for(M, 128), 128, 0, m->stream>>>(m->d_inf, X, M, y);
    M_CUDA(cudaGetLastError());
    return VG_OK;
}

vg_status vg_mlp_features(vg_ctx *c, float *X, int on_device) {
    if (!c) return VG_ERR_ARG;
    if (!c->inserted) return cfail(c, VG_ERR_STATE, "nothing inserted");
    if (!X) return cfail(c, VG_ERR_ARG, "X is NULL");
    const long long B = c->total_blk;
    float *dst = X;
    float *tmp = nullptr;
    if (!on_device) {
        C_CUDA(cudaMalloc((void **)&tmp, sizeof(float) * B * NIN));
        dst = tmp;
    }
    ++g_launch_count;
    k_features<<<nblocks_for(B, 128), 128, 0, c->stream>>>(c->d_sys, (int)c->sys.size(), c->d_bstart, B, dst);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && tmp) {
        e = cudaMemcpyAsync(X, tmp, sizeof(float) * B * NIN, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) return ccuda(c, e, "k_features");
    return VG_OK;
}

}  // extern "C"

namespace {

// k* of every cell of the last compute into c->d_kstar.
vg_status labels_on_device(vg_ctx *c) {
    if (!c->computed) return cfail(c, VG_ERR_STATE, "no computed cells");
    const long long n = c->n;
    C_CUDA(grow(c->d_kstar, c->cap_kstar, n));
    if (n == 0) return VG_OK;
    const int T = 256;
    const long long warps = std::min<long long>(n, (long long)c->sm_count * 64);
    ++g_launch_count;
    k_kstar<<<nblocks_for(warps * 32, T), T, 0, c->stream>>>(c->d_sys, c->d_p64, c->d_sid, c->d_sblk, c->d_ssys,
                                                              c->d_bstart, c->d_rfin, (int)c->sys.size(), n,
                                                              c->d_kstar);
    C_CUDA(cudaGetLastError());
    return VG_OK;
}

}  // namespace

extern "C" {

vg_status vg_mlp_labels(vg_ctx *c, int32_t *kstar, int on_device) {
    if (!c) return VG_ERR_ARG;
    if (c->graph_unchecked) {
        vg_status s = vg_graph_sync(c);
        if (s != VG_OK) return s;
    }
    vg_status s = labels_on_device(c);
    if (s != VG_OK) return s;
    if (!kstar || c->n == 0) return VG_OK;
    C_CUDA(cudaMemcpyAsync(kstar, c->d_kstar, sizeof(int) * c->n,
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    if (!on_device) C_CUDA(cudaStreamSynchronize(c->stream));
    return VG_OK;
}

vg_status vg_mlp_dataset(vg_ctx *c, float *X, float *t, int64_t *m_out) {
    if (!c) return VG_ERR_ARG;
    if (!X || !t || !m_out) return cfail(c, VG_ERR_ARG, "NULL output");
    if (c->graph_unchecked) {
        vg_status s = vg_graph_sync(c);
        if (s != VG_OK) return s;
    }
    vg_status s = labels_on_device(c);
    if (s != VG_OK) return s;
    const long long B = c->total_blk, n = c->n;
    C_CUDA(grow(c->d_kmax, c->cap_kmax, B + 1));
    C_CUDA(grow(c->d_feat, c->cap_feat, B * NIN));
    int *d_flag = nullptr, *d_pos = nullptr;
    C_CUDA(cudaMalloc((void **)&d_flag, sizeof(int) * (B + 1)));
    cudaError_t e = cudaMalloc((void **)&d_pos, sizeof(int) * (B + 1));
    const int T = 256;
    if (e == cudaSuccess) {
        ++g_launch_count;
        k_fill<<<nblocks_for(B, T), T, 0, c->stream>>>(c->d_kmax, B, -1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && n > 0) {
        ++g_launch_count;
        k_block_max<<<nblocks_for(n, T), T, 0, c->stream>>>(c->d_sid, c->d_sblk, c->d_kstar, n, c->d_kmax);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        ++g_launch_count;
        k_features<<<nblocks_for(B, 128), 128, 0, c->stream>>>(c->d_sys, (int)c->sys.size(), c->d_bstart, B,
                                                               c->d_feat);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        ++g_launch_count;
        k_flags<<<nblocks_for(B, T), T, 0, c->stream>>>(c->d_kmax, B, d_flag);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = exclusive_scan_i32(d_flag, d_pos, B, c->d_scan, c->stream);
    if (e == cudaSuccess) {
        ++g_launch_count;
        k_gather_rows<<<nblocks_for(B, T), T, 0, c->stream>>>(c->d_feat, c->d_kmax, d_pos, B, X, t);
        e = cudaGetLastError();
    }
    int last[2] = {0, 0};
    if (e == cudaSuccess && B > 0) e = cudaMemcpyAsync(&last[0], d_pos + B - 1, sizeof(int), cudaMemcpyDeviceToHost,
                                                       c->stream);
    if (e == cudaSuccess && B > 0) e = cudaMemcpyAsync(&last[1], d_flag + B - 1, sizeof(int), cudaMemcpyDeviceToHost,
                                                       c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d_flag);
    if (d_pos) cudaFree(d_pos);
    if (e != cudaSuccess) return ccuda(c, e, "vg_mlp_dataset");
    *m_out = (int64_t)last[0] + last[1];
    return VG_OK;
}

vg_status vg_mlp_predict(vg_ctx *c, vg_mlp *m, float alpha, float kmin, float kmax) {
    if (!c) return VG_ERR_ARG;
    if (!m) return cfail(c, VG_ERR_ARG, "predictor is NULL");
    if (!c->inserted) return cfail(c, VG_ERR_STATE, "nothing inserted");
    if (!(alpha > 0.f) || !(kmin > 0.f) || !(kmax >= kmin)) return cfail(c, VG_ERR_ARG, "alpha, kmin, kmax");
    const long long B = c->total_blk;
    C_CUDA(grow(c->d_kblock, c->cap_kblock, B));
    // the predictor's weights are written on its own stream
    C_CUDA(cudaStreamSynchronize(m->stream));
    C_CUDA(launch_predict(m->d_inf, c->d_sys, (int)c->sys.size(), c->d_bstart, B, alpha, kmin, kmax, c->d_kblock,
                          c->stream));
    c->launches += 1;
    c->kblock_valid = 1;
    return VG_OK;
}

vg_status vg_set_predictor(vg_ctx *c, vg_mlp *m, float alpha, float kmin, float kmax) {
    if (!c) return VG_ERR_ARG;
    if (m && (!(alpha > 0.f) || !(kmin > 0.f) || !(kmax >= kmin))) return cfail(c, VG_ERR_ARG, "alpha, kmin, kmax");
    // the predictor's weights are written on its own stream
    if (m) C_CUDA(cudaStreamSynchronize(m->stream));
    c->pred = m;
    c->pred_alpha = alpha;
    c->pred_kmin = kmin;
    c->pred_kmax = kmax;
    return VG_OK;
}

}  // extern "C"
