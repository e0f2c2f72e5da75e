// Weinberg codes (Sec. 4) of the cells' edge graphs, one warp per cell.
//
// The cell kernel keeps each cell's triangles (plane triples, one per
// vertex, consistently oriented); the top byte of a triangle names the
// earlier slot whose vertex it coincides with (cells of an exact lattice,
// where four or more planes meet at a point, hold several triangles at one
// point).  Darts of the triangulation: vertex v with planes (a, b, c) leaves
// along its three edges, dart 3v + k for the plane pairs (a, b), (b, c),
// (c, a); the edge (x, y) leads to the vertex holding the reverse pair
// (y, x), and dart 3v + k is followed by 3v + (k + 1) mod 3 around v.
//
// The edge graph of the cell merges coincident vertices: a dart between two
// of them has length zero and is contracted.  Around a merged vertex the
// rotation passes a contracted dart by continuing after its reverse, at the
// vertex on its other end (the two rotations are spliced).  A face left
// with two edges (a plane that touches the finished cell along one edge)
// is removed: its two edges become one, whose darts are the reverses of the
// removed face's darts, and the removed darts leave the rotations.
//
// Weinberg's traversal from a start dart: at a new vertex leave by the dart
// after the reverse of the arriving one; at an old vertex return along the
// reverse if it is untraversed, else leave by the first untraversed dart
// after it.  The code lists the labels (order of first visit, from 1) of
// the start and of every arrival: 2E + 1 entries.  The cell's code is the
// lexicographic minimum over every start dart and both rotation directions.
// Every (start, direction) first runs 8 steps, 32 at a time; the minimal
// code begins with the minimal 8-label prefix, so only the starts that have
// it are traced in full.  Those run 32 at a time in lockstep; at every step
// the lanes above the warp's minimum label drop, and the survivors are
// compared with the best code of earlier rounds as they go, so no lane
// stores a code.
// Outputs: darts traversed (2E; 0 = no code), an FNV-1a 64 hash of the
// minimal code (labels as two little-endian bytes each) and the number of
// (start, orientation) pairs that reach it.
#include "vg_internal.cuh"

namespace vg {
namespace {

constexpr int WB_V = 64;            // vertices of a tier-0 cell
constexpr int WB_D = 3 * WB_V;      // darts
constexpr int WB_WARPS = 4;
constexpr int WB_PL = 8;            // labels in a start's prefix key
constexpr unsigned WB_EMPTY = 0xffffffffu;

struct WbSmem {
    unsigned char pair[WB_V][WB_V];  // vertex holding the directed plane pair (x, y)
    unsigned tri[WB_V];              // compacted triangles (plane ids only)
    unsigned char cmap[WB_V];        // slot -> compacted index
    unsigned char cl[WB_V];          // merged vertex of each vertex (its first vertex)
    unsigned char dto[WB_D];         // head vertex of each dart
    unsigned char drev[WB_D];        // reverse dart
    unsigned char rotn[WB_D];        // next dart around the merged tail vertex
    unsigned char rotp[WB_D];        // previous dart around it
    unsigned char mlist[WB_D];       // the darts that are not contracted
    unsigned char dead[WB_D];        // darts of a removed two-edge face
    unsigned char frev[WB_D];        // reverse, rotations and list after the removal
    unsigned char frotn[WB_D];
    unsigned char frotp[WB_D];
    unsigned char flist[WB_D];
    // per lane: labels of merged vertices and the darts traversed; the rows
    // are padded to an odd number of words, so that the lanes of a warp,
    // each in its own row, fall in different shared-memory banks
    unsigned char lab[32][WB_V + 4];
    unsigned used[32][WB_D / 32 + 1];
    unsigned short best[WB_D + 1];   // best code so far
};

__device__ __forceinline__ int dnext(int e) { return e - e % 3 + (e % 3 + 1) % 3; }
__device__ __forceinline__ int dprev(int e) { return e - e % 3 + (e % 3 + 2) % 3; }

__global__ void __launch_bounds__(32 * WB_WARPS) k_weinberg(const unsigned *__restrict__ topo,
                                                            const int *__restrict__ topo_n, long long n,
                                                            int *__restrict__ wlen,
                                                            unsigned long long *__restrict__ whash,
                                                            int *__restrict__ wsym) {
    extern __shared__ __align__(16) unsigned char wb_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1;
    WbSmem &S = reinterpret_cast<WbSmem *>(wb_raw)[warp];
    const long long stride = (long long)gridDim.x * WB_WARPS;
    for (long long cell = (long long)blockIdx.x * WB_WARPS + warp; cell < n; cell += stride) {
        const int nt = topo_n[cell];
        int Dm = 0, sym = 0;
        bool ok = nt > 0 && nt <= WB_V;
        int V = 0;
        if (ok) {
            // compact the occupied slots
            unsigned traw[WB_V / 32];
            int tidx[WB_V / 32];
#pragma unroll
            for (int r = 0; r < WB_V / 32; r++) {
                const unsigned t = topo[cell * WB_V + r * 32 + lane];
                const bool occ = t != WB_EMPTY;
                const unsigned m = __ballot_sync(FULL, occ);
                traw[r] = t;
                tidx[r] = V + __popc(m & lt);
                if (occ) {
                    S.tri[tidx[r]] = t & 0xffffffu;
                    S.cmap[r * 32 + lane] = (unsigned char)tidx[r];
                }
                V += __popc(m);
            }
            ok = V == nt;
            __syncwarp();
            // merged vertices: each vertex points at the earlier one it
            // coincides with; pointer jumping reaches the first of its group
            bool bad = false;
#pragma unroll
            for (int r = 0; r < WB_V / 32; r++) {
                if (traw[r] != WB_EMPTY) {
                    const int into = (int)(traw[r] >> 24);  // 1 + slot, 0 = none
                    int par = tidx[r];
                    if (into > 0) {
                        const int slot = into - 1;
                        if (slot < r * 32 + lane && topo[cell * WB_V + slot] != WB_EMPTY) par = S.cmap[slot];
                        else bad = true;
                    }
                    S.cl[tidx[r]] = (unsigned char)par;
                }
            }
            __syncwarp();
#pragma unroll 1
            for (int it = 0; it < 6; it++) {
                int c2[WB_V / 32];
#pragma unroll
                for (int r = 0; r < WB_V / 32; r++) {
                    const int v = r * 32 + lane;
                    c2[r] = v < V ? S.cl[S.cl[v]] : 0;
                }
                __syncwarp();
#pragma unroll
                for (int r = 0; r < WB_V / 32; r++) {
                    const int v = r * 32 + lane;
                    if (v < V) S.cl[v] = (unsigned char)c2[r];
                }
                __syncwarp();
            }
            // plane pairs -> vertex; every pair of a valid cell is written once
            for (int v = lane; v < V; v += 32) {
                const unsigned t = S.tri[v];
                const int a = t & 0xff, b = (t >> 8) & 0xff, c = (t >> 16) & 0xff;
                if (a < WB_V && b < WB_V && c < WB_V) {
                    S.pair[a][b] = (unsigned char)v;
                    S.pair[b][c] = (unsigned char)v;
                    S.pair[c][a] = (unsigned char)v;
                } else {
                    bad = true;
                }
            }
            __syncwarp();
            const int D = 3 * V;
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
            if (ok) {
                // the darts that join two merged vertices
                for (int d0 = 0; d0 < D; d0 += 32) {
                    const int d = d0 + lane;
                    const bool keep = d < D && S.cl[S.dto[d]] != S.cl[d / 3];
                    const unsigned m = __ballot_sync(FULL, keep);
                    if (keep) S.mlist[Dm + __popc(m & lt)] = (unsigned char)d;
                    Dm += __popc(m);
                }
                __syncwarp();
                // rotations around merged vertices: pass each contracted dart
                // by continuing after its reverse
                for (int j = lane; j < Dm; j += 32) {
                    const int d = S.mlist[j];
                    int e = dnext(d), steps = 0;
                    while (S.cl[S.dto[e]] == S.cl[e / 3] && steps < D) { e = dnext(S.drev[e]); steps++; }
                    int f = dprev(d), fsteps = 0;
                    while (S.cl[S.dto[f]] == S.cl[f / 3] && fsteps < D) { f = dprev(S.drev[f]); fsteps++; }
                    if (steps >= D || fsteps >= D) bad = true;
                    S.rotn[d] = (unsigned char)e;
                    S.rotp[d] = (unsigned char)f;
                }
                __syncwarp();
                ok = Dm > 0 && !__any_sync(FULL, bad);
                // faces of two edges: the successor along a face (rotn of the
                // reverse) returns to the dart in two steps
                if (ok) {
                    for (int j = lane; j < Dm; j += 32) {
                        const int d = S.mlist[j];
                        const int f1 = S.rotn[S.drev[d]];
                        S.dead[d] = S.rotn[S.drev[f1]] == d ? 1 : 0;
                    }
                    __syncwarp();
                    int nlive = 0;
                    for (int j0 = 0; j0 < Dm; j0 += 32) {
                        const int j = j0 + lane;
                        const int d = j < Dm ? S.mlist[j] : 0;
                        const bool live = j < Dm && !S.dead[d];
                        if (live) {
                            // the reverse across removed faces, the rotations
                            // without their darts
                            int r = S.drev[d], g1 = 0;
                            while (S.dead[r] && g1 < Dm) { r = S.drev[S.rotn[S.drev[r]]]; g1++; }
                            int e = S.rotn[d], g2 = 0;
                            while (S.dead[e] && g2 < Dm) { e = S.rotn[e]; g2++; }
                            int f = S.rotp[d], g3 = 0;
                            while (S.dead[f] && g3 < Dm) { f = S.rotp[f]; g3++; }
                            if (g1 >= Dm || g2 >= Dm || g3 >= Dm) bad = true;
                            S.frev[d] = (unsigned char)r;
                            S.frotn[d] = (unsigned char)e;
                            S.frotp[d] = (unsigned char)f;
                        }
                        const unsigned m = __ballot_sync(FULL, live);
                        if (live) S.flist[nlive + __popc(m & lt)] = (unsigned char)d;
                        nlive += __popc(m);
                    }
                    Dm = nlive;
                    __syncwarp();
                    ok = Dm > 0 && !__any_sync(FULL, bad);
                    // none left after the removal
                    if (ok) {
                        for (int j = lane; j < Dm; j += 32) {
                            const int d = S.flist[j];
                            const int f1 = S.frotn[S.frev[d]];
                            if (S.frotn[S.frev[f1]] == d) bad = true;
                        }
                        ok = !__any_sync(FULL, bad);
                    }
                }
            }
        }
        if (ok) {
            bool have = false, stuck = false;
            const int NT = 2 * Dm;
            // one step of a traversal in direction o: mark dart d, label its
            // head, choose the next dart (-1: none left)
            auto step = [&](int d, int o, int &nl, int &L, int &nd) {
                S.used[lane][d >> 5] |= 1u << (d & 31);
                const int y = S.cl[S.dto[d]], rv = S.frev[d];
                const unsigned char *rot = o ? S.frotp : S.frotn;
                nd = -1;
                if (!S.lab[lane][y]) {
                    S.lab[lane][y] = (unsigned char)(++nl);
                    L = nl;
                    nd = rot[rv];
                } else {
                    L = S.lab[lane][y];
                    if (!((S.used[lane][rv >> 5] >> (rv & 31)) & 1)) {
                        nd = rv;
                    } else {
                        int e = rot[rv];
                        for (int guard = 0; ((S.used[lane][e >> 5] >> (e & 31)) & 1) && e != rv && guard < Dm; guard++)
                            e = rot[e];
                        if (!((S.used[lane][e >> 5] >> (e & 31)) & 1)) nd = e;
                    }
                }
            };
            auto reset = [&](int d) {
                for (int v = 0; v < WB_V; v += 4) *reinterpret_cast<unsigned *>(&S.lab[lane][v]) = 0u;
#pragma unroll
                for (int w = 0; w < WB_D / 32; w++) S.used[lane][w] = 0u;
                S.lab[lane][S.cl[d / 3]] = 1;
            };
            // phase 1: the first WB_PL labels of every (start dart, direction),
            // as a key (first label most significant).  The minimal code starts
            // with the minimal key, so only the starts that have it are traced
            // in full.  Keys and the start list use the plane-pair table's
            // storage, free once the dart tables are built.
            unsigned *khi = reinterpret_cast<unsigned *>(&S.pair[0][0]);
            unsigned *klo = khi + 2 * WB_D;
            unsigned short *slist = reinterpret_cast<unsigned short *>(klo + 2 * WB_D);
            for (int r0 = 0; r0 < NT; r0 += 32) {
                const int q = r0 + lane;
                const bool act = q < NT;
                const int o = q >= Dm ? 1 : 0;
                int d = S.flist[act ? q % Dm : 0];
                reset(d);
                __syncwarp();
                int nl = 1;
                unsigned hi = 0, lo = 0;
                bool live = act;
#pragma unroll 1
                for (int k = 0; k < WB_PL; k++) {
                    int L = 0xff, nd = -1;
                    if (live && k < Dm) {
                        step(d, o, nl, L, nd);
                        if (nd >= 0) d = nd; else live = false;
                    }
                    const unsigned b = (unsigned)min(L, 0xff);
                    if (k < 4) hi |= b << (24 - 8 * k);
                    else lo |= b << (24 - 8 * (k - 4));
                }
                if (act) { khi[q] = hi; klo[q] = lo; }
                __syncwarp();
            }
            // the minimal key and the starts that have it
            unsigned mh = 0xffffffffu, ml = 0xffffffffu;
            for (int q = lane; q < NT; q += 32) {
                const unsigned h = khi[q], l = klo[q];
                if (h < mh || (h == mh && l < ml)) { mh = h; ml = l; }
            }
            const unsigned gmh = __reduce_min_sync(FULL, mh);
            const unsigned gml = __reduce_min_sync(FULL, mh == gmh ? ml : 0xffffffffu);
            int NS = 0;
            for (int r0 = 0; r0 < NT; r0 += 32) {
                const int q = r0 + lane;
                const bool keep = q < NT && khi[q] == gmh && klo[q] == gml;
                const unsigned m = __ballot_sync(FULL, keep);
                if (keep) slist[NS + __popc(m & lt)] = (unsigned short)q;
                NS += __popc(m);
            }
            __syncwarp();
            // phase 2: those starts in full, 32 at a time in lockstep
            for (int r0 = 0; r0 < NS; r0 += 32) {
                const int j = r0 + lane;
                bool active = j < NS;
                const int q = slist[active ? j : 0];
                const int o = q >= Dm ? 1 : 0;  // rotation direction
                int d = S.flist[q % Dm];
                reset(d);
                int nl = 1;
                int cmp = have ? 0 : -1;  // 0: equal to the best so far, -1: below it
                if (!have && lane == 0) S.best[0] = 1;
                __syncwarp();
                for (int k = 0; k < Dm; k++) {
                    int L = 0xffff, nd = -1;
                    if (active) {
                        step(d, o, nl, L, nd);
                        if (k + 1 < Dm && nd < 0) stuck = true;
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
                for (int k = 0; k <= Dm; k++) {
                    h ^= (unsigned long long)(S.best[k] & 0xff);
                    h *= 1099511628211ull;
                    h ^= (unsigned long long)(S.best[k] >> 8);
                    h *= 1099511628211ull;
                }
                wlen[cell] = Dm; whash[cell] = h; wsym[cell] = sym;
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
