// Weinberg codes (Sec. 4) of the cells' edge graphs, one warp per cell.
//
// The cell kernel keeps each simple cell's triangles (plane triples, one per
// vertex, consistently oriented).  Darts: vertex v with planes (a, b, c)
// leaves along its three edges, dart 3v + k for the plane pairs (a, b),
// (b, c), (c, a); the edge (x, y) leads to the vertex holding the reverse
// pair (y, x).  Rotation: dart 3v + k is followed by 3v + (k + 1) mod 3.
//
// Weinberg's traversal from a start dart: at a new vertex leave by the dart
// after the reverse of the arriving one; at an old vertex return along the
// reverse if it is untraversed, else leave by the first untraversed dart
// after it.  The code lists the labels (order of first visit, from 1) of
// the start and of every arrival: 2E + 1 entries.  The cell's code is the
// lexicographic minimum over every start dart and both rotation directions.
// The 32 lanes run 32 traversals in lockstep; at every step the lanes above
// the warp's minimum label drop, and the survivors are compared with the
// best code of earlier rounds as they go, so no lane stores a code.
// Outputs: darts traversed (2E; 0 = no code), an FNV-1a 64 hash of the
// minimal code (labels as two little-endian bytes each) and the number of
// (start, orientation) pairs that reach it.
#include "vg_internal.cuh"

namespace vg {
namespace {

constexpr int WB_V = 64;            // vertices of a tier-0 cell
constexpr int WB_D = 3 * WB_V;      // darts
constexpr int WB_WARPS = 4;

struct WbSmem {
    unsigned char pair[WB_V][WB_V];  // vertex holding the directed plane pair (x, y)
    unsigned tri[WB_V];              // compacted triangles
    unsigned char dto[WB_D];         // head vertex of each dart
    unsigned char drev[WB_D];        // reverse dart
    unsigned char lab[32][WB_V];     // per lane: vertex labels of its traversal
    unsigned used[32][WB_D / 32];    // per lane: darts traversed
    unsigned short best[WB_D + 1];   // best code so far
};

__global__ void __launch_bounds__(32 * WB_WARPS) k_weinberg(const unsigned *__restrict__ topo,
                                                            const int *__restrict__ topo_n, long long n,
                                                            int *__restrict__ wlen,
                                                            unsigned long long *__restrict__ whash,
                                                            int *__restrict__ wsym) {
    extern __shared__ __align__(16) unsigned char wb_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WbSmem &S = reinterpret_cast<WbSmem *>(wb_raw)[warp];
    const long long stride = (long long)gridDim.x * WB_WARPS;
    for (long long cell = (long long)blockIdx.x * WB_WARPS + warp; cell < n; cell += stride) {
        const int nt = topo_n[cell];
        int D = 0, sym = 0;
        bool ok = nt > 0 && nt <= WB_V;
        int V = 0;
        if (ok) {
            // compact the occupied slots
#pragma unroll
            for (int r = 0; r < WB_V / 32; r++) {
                const unsigned t = topo[cell * WB_V + r * 32 + lane];
                const bool occ = t != 0xffffffffu;
                const unsigned m = __ballot_sync(FULL, occ);
                if (occ) S.tri[V + __popc(m & ((1u << lane) - 1))] = t;
                V += __popc(m);
            }
            ok = V == nt;
            __syncwarp();
            // plane pairs -> vertex; every pair of a valid cell is written once
            for (int v = lane; v < V; v += 32) {
                const unsigned t = S.tri[v];
                const int a = t & 0xff, b = (t >> 8) & 0xff, c = (t >> 16) & 0xff;
                if (a < WB_V && b < WB_V && c < WB_V) {
                    S.pair[a][b] = (unsigned char)v;
                    S.pair[b][c] = (unsigned char)v;
                    S.pair[c][a] = (unsigned char)v;
                }
            }
            __syncwarp();
            D = 3 * V;
            bool bad = false;
            for (int d = lane; d < D; d += 32) {
                const unsigned t = S.tri[d / 3];
                const int p[3] = {(int)(t & 0xff), (int)((t >> 8) & 0xff), (int)((t >> 16) & 0xff)};
                const int k = d % 3, x = p[k], y = p[(k + 1) % 3];
                if (x >= WB_V || y >= WB_V) { bad = true; continue; }
                const int u = S.pair[y][x];
                int kr = -1;
                if (u < V) {
                    const unsigned tu = S.tri[u];
                    const int q[3] = {(int)(tu & 0xff), (int)((tu >> 8) & 0xff), (int)((tu >> 16) & 0xff)};
#pragma unroll
                    for (int j = 0; j < 3; j++)
                        if (q[j] == y && q[(j + 1) % 3] == x) kr = j;
                }
                if (kr < 0) { bad = true; continue; }
                S.dto[d] = (unsigned char)u;
                S.drev[d] = (unsigned char)(3 * u + kr);
            }
            ok = ok && !__any_sync(FULL, bad);
            __syncwarp();
        }
        if (ok) {
            bool have = false, stuck = false;
            const int NT = 2 * D;
            for (int r0 = 0; r0 < NT; r0 += 32) {
                const int q = r0 + lane;
                bool active = q < NT;
                const int o = q >= D ? 1 : 0;  // rotation direction
                int d = active ? q % D : 0;
                for (int v = 0; v < WB_V; v += 4) *reinterpret_cast<unsigned *>(&S.lab[lane][v]) = 0u;
#pragma unroll
                for (int w = 0; w < WB_D / 32; w++) S.used[lane][w] = 0u;
                int nl = 1;
                S.lab[lane][d / 3] = 1;
                int cmp = have ? 0 : -1;  // 0: equal to the best so far, -1: below it
                if (!have && lane == 0) S.best[0] = 1;
                __syncwarp();
                for (int k = 0; k < D; k++) {
                    int L = 0xffff, nd = -1;
                    if (active) {
                        S.used[lane][d >> 5] |= 1u << (d & 31);
                        const int y = S.dto[d], rv = S.drev[d];
                        // the darts leaving y are base .. base + 2, in rotation order
                        const int base = 3 * (rv / 3);
                        auto R = [&](int e) { return base + (o ? (e - base + 2) % 3 : (e - base + 1) % 3); };
                        if (!S.lab[lane][y]) {
                            S.lab[lane][y] = (unsigned char)(++nl);
                            L = nl;
                            nd = R(rv);
                        } else {
                            L = S.lab[lane][y];
                            if (!((S.used[lane][rv >> 5] >> (rv & 31)) & 1)) {
                                nd = rv;
                            } else {
                                int e = R(rv);
                                while (((S.used[lane][e >> 5] >> (e & 31)) & 1) && e != rv) e = R(e);
                                if (!((S.used[lane][e >> 5] >> (e & 31)) & 1)) nd = e;
                            }
                        }
                        if (k + 1 < D && nd < 0) stuck = true;
                    }
                    const unsigned m = __reduce_min_sync(FULL, (unsigned)L);
                    const unsigned bk = cmp == 0 ? S.best[k + 1] : 0u;
                    __syncwarp();
                    if (cmp == 0) {
                        if (m > bk) { active = false; }
                        else if (m < bk) cmp = -1;
                    }
                    if (!__any_sync(FULL, active)) break;
                    if (cmp == -1 && lane == 0) S.best[k + 1] = (unsigned short)m;
                    active = active && (unsigned)L == m;
                    if (nd >= 0) d = nd;
                    __syncwarp();
                }
                const int surv = __popc(__ballot_sync(FULL, active));
                if (surv > 0) {
                    if (cmp == -1) { sym = surv; have = true; }
                    else sym += surv;
                }
                __syncwarp();
            }
            ok = !__any_sync(FULL, stuck) && have;
        }
        if (lane == 0) {
            if (ok) {
                unsigned long long h = 14695981039346656037ull;
                for (int k = 0; k <= D; k++) {
                    h ^= (unsigned long long)(S.best[k] & 0xff);
                    h *= 1099511628211ull;
                    h ^= (unsigned long long)(S.best[k] >> 8);
                    h *= 1099511628211ull;
                }
                wlen[cell] = D; whash[cell] = h; wsym[cell] = sym;
            } else {
                wlen[cell] = 0; whash[cell] = 0ull; wsym[cell] = 0;
            }
        }
        __syncwarp();
    }
}

}  // namespace

cudaError_t launch_weinberg(const unsigned *topo, const int *topo_n, long long n, int *wlen,
                            unsigned long long *whash, int *wsym, int sm_count, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const size_t smem = sizeof(WbSmem) * WB_WARPS;
    cudaError_t e = cudaFuncSetAttribute(k_weinberg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_weinberg, 32 * WB_WARPS, smem);
    if (e != cudaSuccess) return e;
    const long long need = (n + WB_WARPS - 1) / WB_WARPS;
    const int grid = (int)std::min<long long>(need, (long long)sm_count * std::max(per_sm, 1));
    ++g_launch_count;
    k_weinberg<<<grid, 32 * WB_WARPS, smem, st>>>(topo, topo_n, n, wlen, whash, wsym);
    return cudaGetLastError();
}

}  // namespace vg
