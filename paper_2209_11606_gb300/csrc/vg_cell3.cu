// 3D cell kernel: one warp per Voronoi cell.
//
// The method is the paper's Sec. 2.1: a cell starts as the container box
// relative to its particle (Eqs. 1-2) and each neighbour at relative
// position q removes the half-space r.q > q.q/2 (Eq. 3; radical form
// r.q > (q.q + r_p^2 - r_q^2)/2).  Neighbours are offered near to far and the
// radius bound of Sec. 2.1.3 (no particle beyond 2R can cut, R = max vertex
// distance) ends the computation.
//
// GPU representation (ours, not the paper's Voro++ edge tables): a convex
// polyhedron whose vertices all have degree 3 is stored in its dual form,
// each vertex being the triple of planes (a, b, c) that meet there, ordered
// counter-clockwise seen from outside -- the representation of Ray, Sokolov,
// Lefebvre and Levy, "Meshless Voronoi on the GPU" (ACM TOG 2018).  Vertex k
// lives in lane k % 32, register slot k / 32, with its position cached next
// to its triple.  A cut:
//   1. classifies every vertex against the plane (one FMA chain per lane and
//      slot; a warp ballot tells whether anything lies outside);
//   2. marks the directed edges of the removed triangles in a bit matrix; an
//      edge (x, y) of a removed triangle whose twin (y, x) is unmarked borders
//      the kept part and yields the new vertex (x, y, new plane);
//   3. compacts kept and new vertices through shared memory with a warp scan
//      and solves the new vertices one per lane.
//
// FP32 form: positions relative to the particle in FP32.  Each vertex carries
// the condition number of its three planes; a vertex whose signed distance to
// a cutting plane lies within tol32 * R * |q| (widened by that condition
// number) is re-solved from its three planes in FP64, from the original FP64
// positions, and classified there -- so every topological decision is the
// FP64 one, and FP64 runs only when a decision needs it.
//
// Candidate order: either the walk of Sec. 2.1.3 (blocks by ascending distance
// bound, 32 blocks set up in parallel per window) or a prefetch: the
// candidates inside a radius rho around the particle are gathered from the
// block grid, sorted by distance and cut in that order; the radius bound
// decides, and a cell whose bound still exceeds rho continues with the walk,
// skipping what the prefetch already offered.
//
// Warp-uniform bookkeeping (the candidate source, per-cell constants that
// only cold paths read) lives in per-warp shared memory rather than in
// registers, to keep the register file for the cell itself.
#include <type_traits>

#include "vg_internal.cuh"

namespace vg {
namespace {

constexpr unsigned TRI_EMPTY = 0xffffffffu;
constexpr int KMAX = 128;         // prefetch list capacity
constexpr int NRUN = 64;          // prefetch gather: runs of contiguous blocks
constexpr int RGMAX = 3;          // prefetch gather: largest block reach per axis
constexpr int NBIN = 8;           // prefetch: radial buckets
constexpr float KAP0 = 4.0f;      // condition number covered by the base FP32 band
constexpr float KAP_MAX2 = 1e8f;  // condition number^2 beyond which a new vertex is solved in FP64
constexpr int MAX_SHELL_EXTRA = 4;
// resident CTAs per SM the register budget is sized for: the hot kernel six
// (80 registers a thread, 9.3 KB of shared memory a warp: 24 warps an SM),
// the general tier-0 kernel five (96 registers), the larger tiers four
#ifndef VG_MINB
#define VG_MINB 5
#endif
#ifndef VG_MINB_HOT
#define VG_MINB_HOT 6
#endif
#ifndef VG_MAXT
#define VG_MAXT 128
#endif
// tier-0 lanes per cell and vertex slots per lane (G * VPL = 64)
#ifndef VG_T0_G
#define VG_T0_G 32
#endif
#define VG_T0_VPL (64 / VG_T0_G)
// branch that almost never runs: keep its code out of the common path
#define VG_RARE(c) __builtin_expect(!!(c), 0)
#ifdef VG_MAXREG
#define VG_BOUNDS __maxnreg__(VG_MAXREG)
#else
#define VG_BOUNDS __launch_bounds__(VG_MAXT, MAXP == 64 ? (HOT ? VG_MINB_HOT : VG_MINB) : 4)
#endif

template <typename T> struct V4T;
template <> struct V4T<float> { using t = float4; };
template <> struct V4T<double> { using t = D4; };

template <typename T> __device__ __forceinline__ typename V4T<T>::t mk4(T x, T y, T z, T w);
template <> __device__ __forceinline__ float4 mk4<float>(float x, float y, float z, float w) {
    return make_float4(x, y, z, w);
}
template <> __device__ __forceinline__ D4 mk4<double>(double x, double y, double z, double w) {
    D4 r;
    r.x = x; r.y = y; r.z = z; r.w = w;
    return r;
}

// Per-cell constants read by the cold FP64 paths.
struct CellC {
    int i;        // sorted index
    int self_id;  // input index
    int b[3];     // home block
    int pad;
    double p[3];  // FP64 position
    double rp;    // radius (radical) or 0
    double rmax;  // largest radius of the cell's system (radical) or 0
    double hc;    // clipped cells: half the cube side, 0 = none
};

// Candidate source, warp-uniform.
struct Src {
    int mode;          // 0 prefetch list, 1 walk list, 2 walk shells, 3 done
    int u, count;      // prefetch list cursor and length
    int e;             // walk: next offset list entry
    int shell, sidx;   // walk: Chebyshev shell and position in it
    int vp, vtot;      // walk: particle cursor over the current window
    int nwin;          // walk: blocks in the current window
    int limit, fell_back;
    int last;          // walk: the current window is the last one
    int nbatch;        // candidate batches loaded for this cell
    float rho2;        // prefetch radius^2 (0: none)
    float lo2;         // the preload holds the candidates with lo2 <= |q|^2 < rho2
    int round;         // hot kernel: 0 first preload, 1 the wider second one
    int rg[3];         // prefetch reach in blocks per axis
};

template <typename T, int VPL, int MAXP, int G, bool HOT>
struct Smem {
    // slot indices in the face walk tables: a byte up to 256 vertices
    using FT = typename std::conditional<(G * VPL > 256), unsigned short, unsigned char>::type;
    typename V4T<T>::t pl[MAXP];  // plane normal (x,y,z) and constant (w), cell frame
    int pref[MAXP];               // neighbour's sorted index, or wall code -1..-6
    int pimg[MAXP];               // packed image shift of the neighbour
    float4 v4[G * VPL];                     // FP32 form: the cell's vertices (x, y, z, kappa); free slots 0
    unsigned E[MAXP][MAXP / 32];  // removed directed edges of one cut (32-bit words: native shared atomics)
    union {
        struct {
            int start[NRUN], j0[NRUN], oxb[NRUN], oyz[NRUN];
        } run;                         // prefetch gather: runs of contiguous blocks
        struct {
            int vstart[G], j0[G], o[G], m[G];
        } win;                         // walk: a window of up to G blocks
    } w;
    union {
        struct {
            float4 q[KMAX];  // candidate position relative to the particle, |q|^2
            int2 r[KMAX];    // sorted index and packed image
            int slot[KMAX];  // sorted order of the slots
        } pf;
        struct {
            unsigned stri[G * VPL];            // the cell's triangles, by slot
            T sx[G * VPL], sy[G * VPL], sz[G * VPL];
            FT ftab[G][MAXP];                  // face walk tables, one row per face of a round
            double dpos[HOT ? 1 : G * VPL][3]; // FP64 vertices (degenerate cells; not in the hot kernel)
        } v;                                   // statistics: the finished cell
    } x;
    FT sfirst[G];              // a triangle of each face of a round
    int elist[G * VPL];        // boundary edges (x | y << 8) of one cut
    typename V4T<T>::t cbq[G];   // the current candidate batch: q and |q|^2, one per lane
    int2 cbr[G];                 //   sorted index and packed image
    T cbrj[G];                   //   radius (radical)
    CellC cc;
    Src src;
    int cnt[6];  // work counters
    Sys sysc;    // descriptor of the system of the current cell
    int sys_id;  // which system sysc holds (-1: none)
};

__device__ __forceinline__ int imgc(int img, int a) { return (int)(signed char)((img >> (8 * a)) & 0xff); }
__device__ __forceinline__ int pack_img(int mx, int my, int mz) {
    return (mx & 0xff) | ((my & 0xff) << 8) | ((mz & 0xff) << 16);
}
// Whether the plane q.r = c may cut the cell whose vertices are mirrored in
// v4: some vertex lies beyond -band (band = tau * kappa, the classification's
// FP32 band), widened by 1 % to cover rounding.  A candidate without such a
// vertex removes nothing now, and nothing after later cuts either (the cell
// only shrinks), so one lane can drop it alone instead of the whole warp
// classifying it; every kept candidate still goes through the exact test.
// A free slot holds (0, 0, 0, 0): it keeps a candidate only if c <= 0 (a
// radical plane that the particle itself lies beyond), which is harmless.
// Member si of the surface of Chebyshev shell s (the (2s+1)^3 cube minus its
// interior): two z faces of (2s+1)^2 blocks, two y faces of (2s+1)(2s-1),
// two x faces of (2s-1)^2.
__device__ __forceinline__ void shell_member(int si, int s, int &ox, int &oy, int &oz) {
    const int wd = 2 * s + 1, fa = wd * wd, fb = wd * (wd - 2), fc = (wd - 2) * (wd - 2);
    if (si < 2 * fa) {
        const int r = si < fa ? si : si - fa;
        oz = si < fa ? -s : s;
        ox = r % wd - s;
        oy = r / wd - s;
    } else if (si < 2 * (fa + fb)) {
        const int t = si - 2 * fa, r = t < fb ? t : t - fb;
        oy = t < fb ? -s : s;
        ox = r % wd - s;
        oz = r / wd - (s - 1);
    } else {
        const int t = si - 2 * (fa + fb), r = t < fc ? t : t - fc;
        ox = t < fc ? -s : s;
        oy = r % (wd - 2) - (s - 1);
        oz = r / (wd - 2) - (s - 1);
    }
}

// Block bound (Sec. 2.1.3): a particle q can cut the cell only if some vertex v
// lies beyond its plane, |q - v|^2 < |v|^2 (radical: + rmax^2 - r_p^2, the
// largest radius bounding r_q), so a block whose box [lo, hi] (relative to
// the particle) meets none of those balls holds no cutting particle.  Each
// ball is widened by sl * kappa (FP32 vertex error) and 1e-4 relative.
__device__ __noinline__ bool block_touches(const float4 *v4, int n, float lo0, float lo1, float lo2, float hi0,
                                           float hi1, float hi2, float extra, float sl) {
    bool m = false;
#pragma unroll 1
    for (int t0 = 0; t0 < n; t0 += 8) {
#pragma unroll
        for (int t = t0; t < t0 + 8; t++) {
            const float4 v = v4[t];
            const float dx = fmaxf(0.f, fmaxf(lo0 - v.x, v.x - hi0));
            const float dy = fmaxf(0.f, fmaxf(lo1 - v.y, v.y - hi1));
            const float dz = fmaxf(0.f, fmaxf(lo2 - v.z, v.z - hi2));
            const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float rv = sqrt_a(fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, extra)))) + sl * v.w;
            m |= d2 < rv * rv * 1.0001f;
        }
    }
    return m;
}

// Only the first n entries are read: the rows of slots that hold any vertex
// (n a multiple of 8).
__device__ __forceinline__ bool may_cut(const float4 *v4, int n, float qx, float qy, float qz, float c, float tau) {
    const float lim = -1.01f * tau;
    bool m = false;
#pragma unroll 1
    for (int t0 = 0; t0 < n; t0 += 8) {
#pragma unroll
        for (int t = t0; t < t0 + 8; t++) {
            const float4 v = v4[t];
            const float d = fmaf(v.x, qx, fmaf(v.y, qy, fmaf(v.z, qz, -c)));
            m |= d >= lim * v.w;
        }
    }
    return m;
}

// FP32 band of a candidate close to the particle (|q| below a tenth of the
// smallest block side, so within the adjacent blocks): on top of tol32 R |q|
// the absolute error of block-relative FP32 positions, at most about
// 2^-24 (5 h) per axis there (both offsets, the block side's own rounding,
// the sums), 6e-7 h_max as a vector, times |v| + 2 |q| <= R + 2 |q| (the
// plane's normal and its constant both carry it).  Far candidates keep the
// relative band alone: there the inputs' error is a few percent of it.
__device__ __forceinline__ float band_close(float tol, float r2, float qq, float eabs) {
    const float R = sqrt_a(r2), rq = sqrt_a(qq);
    return tol * R * rq + eabs * (R + 2.f * rq);
}

// prefetch bucket b holds the distances t * rho with t^(3/2) in [b, b+1) / NBIN:
// its lower bound is t = (b / NBIN)^(2/3)
__constant__ float bucket_t[NBIN] = {0.f, 0.25f, 0.396850263f, 0.520020956f,
                                     0.629960525f, 0.731004435f, 0.825481812f, 0.914826428f};
static_assert(NBIN == 8, "bucket_t holds NBIN = 8 bounds");

__device__ __forceinline__ int tri_a(unsigned t) { return t & 0xff; }
__device__ __forceinline__ int tri_b(unsigned t) { return (t >> 8) & 0xff; }
__device__ __forceinline__ int tri_c(unsigned t) { return (t >> 16) & 0xff; }
__device__ __forceinline__ unsigned mk_tri(int a, int b, int c) {
    return (unsigned)a | ((unsigned)b << 8) | ((unsigned)c << 16);
}

// Group primitives: a cell is handled by G consecutive lanes (G = 32: one
// warp per cell; G = 16: two cells per warp).  gmask holds the group's lanes;
// lane indices below are relative to the group.
template <int G>
__device__ __forceinline__ unsigned gballot(unsigned gmask, int gbase, bool p) {
    const unsigned b = __ballot_sync(gmask, p);
    if constexpr (G == 32) return b;
    else return (b >> gbase) & ((1u << G) - 1);
}
template <int G>
__device__ __forceinline__ int gexcl_scan(unsigned gmask, int v, int gl, int &total) {
    int x = v;
#pragma unroll
    for (int d = 1; d < G; d <<= 1) {
        int y = __shfl_up_sync(gmask, x, d, G);
        if (gl >= d) x += y;
    }
    total = __shfl_sync(gmask, x, G - 1, G);
    return x - v;
}
template <int G>
__device__ __forceinline__ double gsum(unsigned gmask, double v) {
#pragma unroll
    for (int d = G / 2; d > 0; d >>= 1) v += __shfl_xor_sync(gmask, v, d, G);
    return v;
}
template <int G>
__device__ __forceinline__ float gsum(unsigned gmask, float v) {
#pragma unroll
    for (int d = G / 2; d > 0; d >>= 1) v += __shfl_xor_sync(gmask, v, d, G);
    return v;
}
template <int G>
__device__ __forceinline__ double gmax(unsigned gmask, double v) {
#pragma unroll
    for (int d = G / 2; d > 0; d >>= 1) v = fmax(v, __shfl_xor_sync(gmask, v, d, G));
    return v;
}
template <int G>
__device__ __forceinline__ float gmax(unsigned gmask, float v) {
    // non-negative floats order like their bit patterns
    return __int_as_float((int)__reduce_max_sync(gmask, (unsigned)__float_as_int(v)));
}
__device__ __forceinline__ unsigned long long gor64(unsigned gmask, unsigned long long v) {
    unsigned lo = __reduce_or_sync(gmask, (unsigned)v);
    unsigned hi = __reduce_or_sync(gmask, (unsigned)(v >> 32));
    return ((unsigned long long)hi << 32) | lo;
}

// Bitonic sort of G keys, one per lane of a group, with the stage loops kept
// rolled (the network runs once per cell; small code matters more).
template <int G>
__device__ __forceinline__ unsigned long long bitonic1(unsigned long long k, int gl, unsigned gmask) {
#pragma unroll 1
    for (int size = 2; size <= G; size <<= 1) {
#pragma unroll 1
        for (int j = size >> 1; j > 0; j >>= 1) {
            const bool up = (gl & size) == 0;
            const unsigned long long ot = __shfl_xor_sync(gmask, k, j, G);
            const bool keep_min = ((gl & j) == 0) == up;
            const unsigned long long mn = k < ot ? k : ot, mx = k < ot ? ot : k;
            k = keep_min ? mn : mx;
        }
    }
    return k;
}

// Bitonic sort of 2G keys, two per lane (element g = 2 gl + e), stage loops
// rolled.
template <int G>
__device__ __forceinline__ void bitonic2(unsigned long long &k0, unsigned long long &k1, int gl, unsigned gmask) {
#pragma unroll 1
    for (int size = 2; size <= 2 * G; size <<= 1) {
#pragma unroll 1
        for (int j = size >> 1; j > 0; j >>= 1) {
            const int g0 = 2 * gl;
            if (j == 1) {
                const bool up = (g0 & size) == 0;
                const bool sw = up ? (k0 > k1) : (k0 < k1);
                if (sw) { const unsigned long long t = k0; k0 = k1; k1 = t; }
            } else {
                const int lm = j >> 1;
                const unsigned long long o0 = __shfl_xor_sync(gmask, k0, lm, G);
                const unsigned long long o1 = __shfl_xor_sync(gmask, k1, lm, G);
                const bool up0 = (g0 & size) == 0, up1 = ((g0 + 1) & size) == 0;
                const bool km0 = ((g0 & j) == 0) == up0, km1 = (((g0 + 1) & j) == 0) == up1;
                k0 = km0 ? (k0 < o0 ? k0 : o0) : (k0 < o0 ? o0 : k0);
                k1 = km1 ? (k1 < o1 ? k1 : o1) : (k1 < o1 ? o1 : k1);
            }
        }
    }
}

// Bitonic sort of G*E keys held E per lane of a group (element g = gl*E + e).
template <int E, int G>
__device__ __forceinline__ void bitonic(unsigned long long (&k)[E], int gl, unsigned gmask) {
#pragma unroll
    for (int size = 2; size <= G * E; size <<= 1) {
#pragma unroll
        for (int j = size >> 1; j > 0; j >>= 1) {
            if (j < E) {
#pragma unroll
                for (int e = 0; e < E; e++) {
                    if ((e & j) == 0) {
                        int gi = gl * E + e;
                        bool up = (gi & size) == 0;
                        unsigned long long a = k[e], b = k[e ^ j];
                        bool sw = up ? (a > b) : (a < b);
                        if (sw) { k[e] = b; k[e ^ j] = a; }
                    }
                }
            } else {
                int lm = j / E;
#pragma unroll
                for (int e = 0; e < E; e++) {
                    int gi = gl * E + e;
                    bool up = (gi & size) == 0;
                    unsigned long long ot = __shfl_xor_sync(gmask, k[e], lm, G);
                    bool lower = (gi & j) == 0;
                    bool keep_min = (lower == up);
                    unsigned long long mn = k[e] < ot ? k[e] : ot, mx = k[e] < ot ? ot : k[e];
                    k[e] = keep_min ? mn : mx;
                }
            }
        }
    }
}

// FP64 plane of a neighbour (sorted index `ref`, image `img`) or of a wall
// (ref = -(1 + 2 axis + side)): the cell lies on n.r <= c, relative to p.
// Same operation order as the oracle's: q = (x_j + m L) - x_p.
__device__ __forceinline__ void plane64(const Grid &g, const Store &s, const CellC &ci, int ref, int img,
                                        double n[3], double &c) {
    if (ref < 0) {
        int w = -ref - 1, a = w >> 1, side = w & 1;
        n[0] = n[1] = n[2] = 0.0;
        n[a] = side ? 1.0 : -1.0;
        c = side ? __dsub_rn(g.hi[a], ci.p[a]) : __dsub_rn(ci.p[a], g.lo[a]);
        // a clipped cell's cube face (on a periodic axis every wall is one)
        if (ci.hc > 0.0 && (g.per[a] || ci.hc < c)) c = ci.hc;
        return;
    }
    D4 q = s.p64[ref];
    double qa[3] = {q.x, q.y, q.z};
    double qq = 0.0;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        n[a] = __dsub_rn(__dadd_rn(qa[a], __dmul_rn((double)imgc(img, a), g.L[a])), ci.p[a]);
        qq = __dadd_rn(qq, __dmul_rn(n[a], n[a]));
    }
    c = __dmul_rn(0.5, __dsub_rn(__dadd_rn(qq, __dmul_rn(ci.rp, ci.rp)), __dmul_rn(q.w, q.w)));
}

// Intersection of three planes by Cramer's rule, FP64.
__device__ __forceinline__ void solve3_d(const double n1[3], double c1, const double n2[3], double c2,
                                         const double n3[3], double c3, double v[3]) {
    double x23[3] = {n2[1] * n3[2] - n2[2] * n3[1], n2[2] * n3[0] - n2[0] * n3[2], n2[0] * n3[1] - n2[1] * n3[0]};
    double x31[3] = {n3[1] * n1[2] - n3[2] * n1[1], n3[2] * n1[0] - n3[0] * n1[2], n3[0] * n1[1] - n3[1] * n1[0]};
    double x12[3] = {n1[1] * n2[2] - n1[2] * n2[1], n1[2] * n2[0] - n1[0] * n2[2], n1[0] * n2[1] - n1[1] * n2[0]};
    double det = n1[0] * x23[0] + n1[1] * x23[1] + n1[2] * x23[2];
    double id = 1.0 / det;
#pragma unroll
    for (int a = 0; a < 3; a++) v[a] = (c1 * x23[a] + c2 * x31[a] + c3 * x12[a]) * id;
}

// ---- cold FP64 paths (out of line) ----------------------------------------------

// FP64 position of the vertex with plane triple t.
__device__ __noinline__ void vertex64(const Grid *g, const Store *st, const CellC *ci, const int *pref,
                                      const int *pimg, unsigned t, double *v) {
    double n1[3], n2[3], n3[3], c1, c2, c3;
    int a = tri_a(t), b = tri_b(t), c = tri_c(t);
    plane64(*g, *st, *ci, pref[a], pimg[a], n1, c1);
    plane64(*g, *st, *ci, pref[b], pimg[b], n2, c2);
    plane64(*g, *st, *ci, pref[c], pimg[c], n3, c3);
    double r[3];
    solve3_d(n1, c1, n2, c2, n3, c3, r);
    v[0] = r[0]; v[1] = r[1]; v[2] = r[2];
}

// FP64 classification of vertex t against the plane of neighbour (ref, img):
// 1 outside, 0 on the plane (|d| <= tau_rel*s*|q|), -1 inside.
__device__ __noinline__ int classify64(const Grid *g, const Store *st, const CellC *ci, const int *pref,
                                       const int *pimg, unsigned t, int ref, int img, double tau_rel_s) {
    double v[3];
    vertex64(g, st, ci, pref, pimg, t, v);
    double q[3], cq;
    plane64(*g, *st, *ci, ref, img, q, cq);
    double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
    double tau = tau_rel_s * qn;
    double d = __dsub_rn(__dadd_rn(__dadd_rn(__dmul_rn(q[0], v[0]), __dmul_rn(q[1], v[1])), __dmul_rn(q[2], v[2])), cq);
    return d > tau ? 1 : (d >= -tau ? 0 : -1);
}

// FP64 solve of the new vertex on planes x, y and the cutting plane.
__device__ __noinline__ float3 solve_new64(const Grid *g, const Store *st, const CellC *ci, const int *pref,
                                           const int *pimg, int x, int y, int ref, int img) {
    double n1[3], n2[3], n3[3], c1, c2, c3, v[3];
    plane64(*g, *st, *ci, pref[x], pimg[x], n1, c1);
    plane64(*g, *st, *ci, pref[y], pimg[y], n2, c2);
    plane64(*g, *st, *ci, ref, img, n3, c3);
    solve3_d(n1, c1, n2, c2, n3, c3, v);
    return make_float3((float)v[0], (float)v[1], (float)v[2]);
}

// ---- geometry of candidates ------------------------------------------------------

// FP32 position of particle pj seen from the cell's particle (offset o0..o2
// in its home block) through block offset (ox, oy, oz); shared by the
// prefetch gather and the walk so that both see bit-identical distances.
__device__ __forceinline__ void cand32(const Grid &g, float o0, float o1, float o2, float4 pj, int ox, int oy,
                                       int oz, float &qx, float &qy, float &qz, float &qq) {
    qx = __fadd_rn(__fmul_rn((float)ox, g.hf[0]), __fsub_rn(pj.x, o0));
    qy = __fadd_rn(__fmul_rn((float)oy, g.hf[1]), __fsub_rn(pj.y, o1));
    qz = __fadd_rn(__fmul_rn((float)oz, g.hf[2]), __fsub_rn(pj.z, o2));
    qq = __fadd_rn(__fadd_rn(__fmul_rn(qx, qx), __fmul_rn(qy, qy)), __fmul_rn(qz, qz));
}

__device__ __forceinline__ void cand64(const Grid &g, const CellC &ci, D4 pj, int mx, int my, int mz, double &qx,
                                       double &qy, double &qz, double &qq) {
    qx = __dsub_rn(__dadd_rn(pj.x, __dmul_rn((double)mx, g.L[0])), ci.p[0]);
    qy = __dsub_rn(__dadd_rn(pj.y, __dmul_rn((double)my, g.L[1])), ci.p[1]);
    qz = __dsub_rn(__dadd_rn(pj.z, __dmul_rn((double)mz, g.L[2])), ci.p[2]);
    qq = __dadd_rn(__dadd_rn(__dmul_rn(qx, qx), __dmul_rn(qy, qy)), __dmul_rn(qz, qz));
}

// Distance from the particle to the slab of block offset o along axis a, FP32.
__device__ __forceinline__ float axis_gap(const Grid &g, float oa, int a, int o) {
    float lo = __fsub_rn(__fmul_rn((float)o, g.hf[a]), oa);
    float hi = __fadd_rn(lo, g.hf[a]);
    return lo > 0.f ? lo : (hi < 0.f ? -hi : 0.f);
}
__device__ __forceinline__ float row_gap2(const Grid &g, float o1, float o2, int oy, int oz) {
    float gy = axis_gap(g, o1, 1, oy), gz = axis_gap(g, o2, 2, oz);
    return __fadd_rn(__fmul_rn(gy, gy), __fmul_rn(gz, gz));
}
__device__ __forceinline__ float block_gap2(const Grid &g, float o0, float o1, float o2, int ox, int oy, int oz) {
    float gx = axis_gap(g, o0, 0, ox);
    return __fadd_rn(__fmul_rn(gx, gx), row_gap2(g, o1, o2, oy, oz));
}

// Block offset o -> global block index (the system's first block `base`
// plus the block inside the system) and image shift; false outside a wall.
__device__ __forceinline__ bool resolve(const Grid &g, long long base, const int *b, int ox, int oy, int oz, int &k,
                                        int &mx, int &my, int &mz) {
    int o[3] = {ox, oy, oz}, t[3], m[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        int ta = b[a] + o[a];
        m[a] = 0;
        if (g.per[a]) {
            m[a] = floordiv_near(ta, g.nb[a]);
            ta -= m[a] * g.nb[a];
        } else if (ta < 0 || ta >= g.nb[a]) {
            return false;
        }
        t[a] = ta;
    }
    k = (int)base + t[0] + g.nb[0] * (t[1] + g.nb[1] * t[2]);
    mx = m[0]; my = m[1]; mz = m[2];
    return true;
}

// Preload radius of every block: the ball that holds the block's candidate
// target at the density of the 27 blocks around it (a block with n27
// particles in v27 blocks inside the box), rho = (3 k / (4 pi dens))^(1/3).
__global__ void k_prefetch_rho(const Sys *__restrict__ sys, int nsys, const int *__restrict__ bstart, long long nblk,
                               const float *__restrict__ kblock, float kfixed, float *__restrict__ rho) {
    const long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (b >= nblk) return;
    int sidx = 0;
    if (nsys > 1) {
        int lo = 0, hi = nsys - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (sys[mid].blk_base <= b) lo = mid; else hi = mid - 1;
        }
        sidx = lo;
    }
    const Sys &sy = sys[sidx];
    const Grid &g = sy.g;
    const long long kl = b - sy.blk_base;
    const int hb[3] = {(int)(kl % g.nb[0]), (int)((kl / g.nb[0]) % g.nb[1]), (int)(kl / ((long long)g.nb[0] * g.nb[1]))};
    int n27 = 0, v27 = 0;
    float lk = 0.f;
    for (int q = 0; q < 27; q++) {
        int kk, mx, my, mz;
        if (resolve(g, sy.blk_base, hb, q % 3 - 1, (q / 3) % 3 - 1, q / 9 - 1, kk, mx, my, mz)) {
            n27 += bstart[kk + 1] - bstart[kk];
            v27 += 1;
            if (kblock) lk += logf(fmaxf(8.f, kblock[kk]));
        }
    }
    // learned targets: the geometric mean over the 27 blocks
    const float kt = kblock ? expf(lk / (float)max(v27, 1)) : kfixed;
    const float dens = (float)max(n27, 1) * rcp_a((float)max(v27, 1) * g.hf[0] * g.hf[1] * g.hf[2]);
    rho[b] = cbrt_a(3.f * kt * rcp_a(4.f * 3.14159265f * dens));
}

// ---- the kernel ------------------------------------------------------------------

// HOT: the common path only (FP32, prefetch, tier 0).  A cell that needs
// anything else -- the walk after both preloads, FP64 vertices for its
// statistics (degenerate, ill-conditioned or thin cells), more than 64
// planes or 32 faces, or a batched system marked for the general kernel --
// is handed on whole, through the deferred list, to the general kernel
// (tier 3), which computes it from the start.  The hot kernel's code then
// holds neither the walk nor the FP64 statistics nor those rare branches,
// which keeps the path it runs compact in the instruction cache.
// (the second preload's label is used by the hot instantiation only)
#pragma nv_diag_suppress 177
template <typename T, int VPL, int MAXP, bool BATCH, int G, bool TOPO = false, bool HOT = false>
__global__ void VG_BOUNDS
    k_cells3(const __grid_constant__ Store st, const __grid_constant__ Out o,
             const __grid_constant__ Params pp, const __grid_constant__ Offsets off, unsigned *ticket,
             const int *cells, int ncells, int tier) {
    constexpr bool F32 = sizeof(T) == 4;
    constexpr int CAP = G * VPL;
    constexpr int NW = MAXP / 64;
    constexpr int R = MAXP / G;
    using S_t = Smem<T, VPL, MAXP, G, HOT>;
    extern __shared__ __align__(32) unsigned char smem_raw[];
    // G lanes per cell: gl is the lane within the cell's group
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gl = lane % G, gbase = lane - gl;
    const unsigned gmask = G == 32 ? FULL : (((1u << G) - 1) << gbase);
    S_t &S = reinterpret_cast<S_t *>(smem_raw)[warp * (32 / G) + lane / G];
    Src &src = S.src;
    // the edge matrix starts clear; every cut leaves it clear
    for (int u = gl; u < MAXP * (MAXP / 32); u += G) (&S.E[0][0])[u] = 0u;
    if (gl == 0) S.sys_id = -1;
    __syncwarp(gmask);
    const Sys &SY = sys_ref<BATCH>(st, S.sysc);
    const Grid &g = SY.g;
    // tier 0 takes all cells (or a caller's subset), tier 3 the cells the hot
    // kernel deferred, tiers 1 and 2 the cells the tier below handed on
    const int total = cells ? (tier == 1 ? *o.retry_count
                                         : (tier == 2 ? *o.retry2_count : (tier == 3 ? *o.retry0_count : ncells)))
                            : st.n;
    const int chunk = pp.chunk > 0 ? pp.chunk : 1;
    // FP32 band factor, converted once (FP64 work is scarce on this part)
    const float tol32f = (float)pp.tol32;

    for (int iter = 0; iter < (1 << 30); iter++) {
        int base = 0;
        if (gl == 0) base = (int)atomicAdd(ticket, (unsigned)chunk);
        base = __shfl_sync(gmask, base, 0, G);
        if (base >= total) break;
        const int wend = min(base + chunk, total);
        for (int w = base; w < wend; w++) {
            const int i = cells ? cells[w] : w;
            // ---------------------------------------------------------- setup
            if constexpr (BATCH) {
                // the cell's system descriptor, kept while consecutive cells share it
                const int sidx = __ldg(&st.ssys[i]);
                if (sidx != S.sys_id) {
                    __syncwarp(gmask);
                    const int *src32 = reinterpret_cast<const int *>(&st.sys[sidx]);
                    int *dst32 = reinterpret_cast<int *>(&S.sysc);
                    for (int u = gl; u < (int)(sizeof(Sys) / 4); u += G) dst32[u] = __ldg(&src32[u]);
                    if (gl == 0) S.sys_id = sidx;
                    __syncwarp(gmask);
                }
                if constexpr (HOT) {
                    // a system marked for the general kernel: all its cells go there
                    if (!S.sysc.hot) {
                        if (gl == 0) {
                            const int slot = atomicAdd(o.retry0_count, 1);
                            o.retry0[slot] = i;
                        }
                        __syncwarp(gmask);
                        continue;
                    }
                }
            }
            const int kh = __ldg(&st.sblk[i]);
            const int khl = kh - (int)SY.blk_base;
            float o0, o1, o2, rp32;
            {
                const float4 p32 = __ldg(&st.p32[i]);
                o0 = p32.x; o1 = p32.y; o2 = p32.z; rp32 = p32.w;
                if (gl == 0) {
                    const D4 p64 = st.p64[i];
                    S.cc.i = i;
                    S.cc.self_id = __ldg(&st.sid[i]);
                    S.cc.b[0] = khl % g.nb[0];
                    S.cc.b[1] = (khl / g.nb[0]) % g.nb[1];
                    S.cc.b[2] = khl / (g.nb[0] * g.nb[1]);
                    S.cc.p[0] = p64.x; S.cc.p[1] = p64.y; S.cc.p[2] = p64.z;
                    S.cc.rp = p64.w;
                    S.cc.rmax = st.radical ? (BATCH ? S.sysc.rmax : st.sys[0].rmax) : 0.0;
                    S.cc.hc = 0.5 * pp.clip;
                }
                if (pp.collect && gl < 6) S.cnt[gl] = 0;  // [5] sums the preloads of both rounds
            }
            // ------------------------------------- initial cell, Eqs. (1)-(2)
            unsigned tri[VPL];
            T vx[VPL], vy[VPL], vz[VPL];
            float kap[VPL];
            {
                __syncwarp(gmask);
                T lo[3], hi[3];
                const float oo[3] = {o0, o1, o2};
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    if (g.per[a]) {
                        if constexpr (F32) { lo[a] = -0.5f * g.Lf[a]; hi[a] = 0.5f * g.Lf[a]; }
                        else { lo[a] = -0.5 * g.L[a]; hi[a] = 0.5 * g.L[a]; }
                    } else if constexpr (F32) {
                        lo[a] = -((float)S.cc.b[a] * g.hf[a] + oo[a]);
                        hi[a] = (float)(g.nb[a] - S.cc.b[a]) * g.hf[a] - oo[a];
                    } else {
                        lo[a] = g.lo[a] - S.cc.p[a];
                        hi[a] = g.hi[a] - S.cc.p[a];
                    }
                }
                // clipped cells (Sec. 3.1.3): the box meets the cube of side clip
                // around the particle; on a periodic axis a cube smaller than the
                // period replaces the self-image planes by walls
                if (VG_RARE(pp.clip > 0.0)) {
                    const T hc = (T)(0.5 * pp.clip);
#pragma unroll
                    for (int a = 0; a < 3; a++) {
                        if (g.per[a]) {
                            if (pp.clip < g.L[a]) { lo[a] = -hc; hi[a] = hc; }
                        } else {
                            lo[a] = lo[a] > -hc ? lo[a] : -hc;
                            hi[a] = hi[a] < hc ? hi[a] : hc;
                        }
                    }
                }
                if (gl < 6) {
                    const int a = gl >> 1, side = gl & 1;
                    T n[3] = {0, 0, 0};
                    T c;
                    int ref, img;
                    if (g.per[a] && !(pp.clip > 0.0 && pp.clip < g.L[a])) {
                        if constexpr (F32) {
                            n[a] = side ? g.Lf[a] : -g.Lf[a];
                            c = 0.5f * g.Lf[a] * g.Lf[a];
                        } else {
                            n[a] = side ? g.L[a] : -g.L[a];
                            c = 0.5 * g.L[a] * g.L[a];
                        }
                        ref = i;
                        img = pack_img(a == 0 ? (side ? 1 : -1) : 0, a == 1 ? (side ? 1 : -1) : 0,
                                       a == 2 ? (side ? 1 : -1) : 0);
                    } else {
                        n[a] = side ? (T)1 : (T)-1;
                        c = side ? hi[a] : -lo[a];
                        ref = -(1 + 2 * a + side);
                        img = 0;
                    }
                    S.pl[gl] = mk4<T>(n[0], n[1], n[2], c);
                    S.pref[gl] = ref;
                    S.pimg[gl] = img;
                }
#pragma unroll
                for (int s = 0; s < VPL; s++) {
                    tri[s] = TRI_EMPTY;
                    vx[s] = vy[s] = vz[s] = (T)0;
                    kap[s] = 1.f;
                }
                if (gl < 8) {
                    const int sx = gl & 1, sy = (gl >> 1) & 1, sz = (gl >> 2) & 1;
                    const int minus = (1 - sx) + (1 - sy) + (1 - sz);
                    const int A = sx, B = 2 + sy, C = 4 + sz;
                    tri[0] = (minus & 1) ? mk_tri(A, C, B) : mk_tri(A, B, C);
                    vx[0] = sx ? hi[0] : lo[0];
                    vy[0] = sy ? hi[1] : lo[1];
                    vz[0] = sz ? hi[2] : lo[2];
                }
                if constexpr (F32) {
#pragma unroll
                    for (int s = 0; s < VPL; s++)
                        S.v4[s * G + gl] = tri[s] != TRI_EMPTY ? make_float4(vx[s], vy[s], vz[s], kap[s])
                                                                  : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            int ntri = 8;        // vertices
            unsigned rows = 1;   // register slots (rows of G lanes) that hold any vertex
            // FP32: the vertex mirror is rebuilt before the next batch reads it,
            // not after every cut (warp-uniform)
            bool mdirty = false;
            // planes in use: a counter hands out plane slots; the exact set of
            // live planes (those some vertex still lies on) is rebuilt from the
            // vertices only when the counter runs out and for the statistics
            unsigned long long live[NW];
#pragma unroll
            for (int w2 = 0; w2 < NW; w2++) live[w2] = w2 == 0 ? 0x3full : 0ull;
            int nplane = 6;
            auto live_planes = [&]() {
                unsigned long long lv[NW];
#pragma unroll
                for (int w2 = 0; w2 < NW; w2++) lv[w2] = 0;
#pragma unroll
                for (int s = 0; s < VPL; s++) {
                    if (tri[s] != TRI_EMPTY) {
                        const int a = tri_a(tri[s]), b = tri_b(tri[s]), cc = tri_c(tri[s]);
                        lv[a >> 6] |= 1ull << (a & 63);
                        lv[b >> 6] |= 1ull << (b & 63);
                        lv[cc >> 6] |= 1ull << (cc & 63);
                    }
                }
#pragma unroll
                for (int w2 = 0; w2 < NW; w2++) live[w2] = gor64(gmask, lv[w2]);
            };
            T r2 = gmax<G>(gmask, gl < 8 ? vx[0] * vx[0] + vy[0] * vy[0] + vz[0] * vz[0] : (T)0);
            // bit 0 degenerate, 1 capacity/consistency failure, 2 empty, 3 duplicate
            // point, 4 a close cut (FP32)
            int flags = 0;
            // FP32: candidates closer than qabs2 take the absolute input error
            // eabs; a cut closer than qclose2 tilts its plane by eabs / |q|, too
            // much for FP32 statistics (bit 4 of flags: FP64 vertices)
            const float hmin3 = fminf(g.hf[0], fminf(g.hf[1], g.hf[2]));
            const float qabs2 = 0.01f * hmin3 * hmin3, qclose2 = 0.0025f * hmin3 * hmin3;
            const float eabs = 6e-7f * fmaxf(g.hf[0], fmaxf(g.hf[1], g.hf[2]));

            // radius bound (Sec. 2.1.3), squared, with a small relative margin
            // that covers the rounding of R and of candidate distances
            // FP32: the inputs' absolute error eabs moves |q| and R by about
            // eabs and the vertices by kappa eabs; 64 eabs R covers a small cell
            // (FP32: approximate roots, a few ulps against the 1e-4 margin)
            auto root = [](T x) -> T {
                if constexpr (F32) return sqrt_a(x);
                else return sqrt(x);
            };
            auto stop2 = [&]() -> T {
                const T margin = F32 ? (T)1.0001 : (T)(1.0 + 1e-12);
                const T ea = F32 ? (T)(64.f * eabs) : (T)0;
                if (!st.radical) return (T)4 * r2 * margin + ea * root(r2);
                T disc = r2 + (T)(S.cc.rmax * S.cc.rmax) - (T)(S.cc.rp * S.cc.rp);
                if (disc <= (T)0) return (T)0;
                T rs = root(r2) + root(disc);
                return rs * rs * margin + ea * rs;
            };

            // ----------------------------------------------- candidate source
            src.mode = 1;
            src.rho2 = 0.f;
            src.rg[0] = src.rg[1] = src.rg[2] = 0;
            src.count = 0;
            src.u = 0;
            src.e = 0;
            src.shell = 1;
            src.sidx = 0;
            src.vp = 0;
            src.vtot = 0;
            src.nwin = 0;
            src.limit = 0;
            src.fell_back = 0;
            src.last = 0;
            src.nbatch = 0;
            src.lo2 = 0.f;
            src.round = 0;
            // the hot kernel's second preload: when the bound reaches past the
            // first one, the candidates of a wider shell are gathered and cut
            // the same way instead of handing the cell on
        regather:
            if constexpr (F32) {
                if (pp.order == VG_PREFETCH && st.n < (1 << 27)) {
                    // the block's preload radius, computed per block before the
                    // launch; a second round reaches past the bound with a margin
                    const float lo2 = src.lo2;
                    float rho = src.round == 0 ? __ldg(&pp.rhoblk[kh])
                                           : fmaxf(1.26f * sqrt_a(lo2), 1.01f * sqrt_a((float)stop2()));
                    int count = 0;
                    bool give_up = false;
                    float rho2 = 0.f;
                    int rg0 = 0, rg1 = 0, rg2 = 0;
#pragma unroll 1
                    for (int attempt = 0; attempt < 6; attempt++) {
                        rho2 = rho * rho;
                        // block reach, rounded up with a margin over the approximate quotient
                        const float rm = rho * 1.0001f;
                        rg0 = (int)ceilf(rm * rcp_a(g.hf[0]));
                        rg1 = (int)ceilf(rm * rcp_a(g.hf[1]));
                        rg2 = (int)ceilf(rm * rcp_a(g.hf[2]));
                        count = 0;
                        if (rg0 > RGMAX || rg1 > RGMAX || rg2 > RGMAX) { give_up = true; break; }
                        // 1. runs of contiguous blocks: rows along x (fixed oy, oz)
                        //    split where the x image shift changes; one row per gl
                        const int wy = 2 * rg1 + 1, nrows = wy * (2 * rg2 + 1);
                        const int bx = S.cc.b[0];
                        int nrun = 0, npart = 0;
#pragma unroll 1
                        for (int r0 = 0; r0 < nrows; r0 += G) {
                            const int r = r0 + gl;
                            int oy = 0, oz = 0, krow = 0, ox = 0, oxhi = -1, myz = 0;
                            bool rowok = false;
                            if (r < nrows) {
                                // r / wy for r < 64, wy <= 7: the approximate quotient of
                                // r + 1/2 is within 0.5 / wy of the exact one
                                const int rq = (int)(((float)r + 0.5f) * rcp_a((float)wy));
                                oy = r - rq * wy - rg1;
                                oz = rq - rg2;
                                int kk, mx, my, mz;
                                rowok = row_gap2(g, o1, o2, oy, oz) < rho2 &&
                                        resolve(g, SY.blk_base, S.cc.b, 0, oy, oz, kk, mx, my, mz);
                                // image shifts are at most RGMAX blocks: 4 bits each
                                myz = ((my + 8) << 20) | ((mz + 8) << 24);
                                krow = kk - bx;
                                if (rowok) {
                                    // the blocks of the row within rho: an interval around 0
                                    int lo = 0, hi = 0;
                                    while (lo > -rg0 && block_gap2(g, o0, o1, o2, lo - 1, oy, oz) < rho2) lo--;
                                    while (hi < rg0 && block_gap2(g, o0, o1, o2, hi + 1, oy, oz) < rho2) hi++;
                                    if (!g.per[0]) { lo = max(lo, -bx); hi = min(hi, g.nb[0] - 1 - bx); }
                                    ox = lo;
                                    oxhi = hi;
                                }
                            }
#pragma unroll 1
                            for (int k = 0; k <= 2 * RGMAX; k++) {
                                bool have = rowok && ox <= oxhi;
                                int xa = 0, xb = 0, m0 = 0;
                                if (have) {
                                    const int tx = bx + ox;
                                    if (g.per[0]) {
                                        m0 = floordiv_near(tx, g.nb[0]);
                                        xa = tx - m0 * g.nb[0];
                                        xb = min(g.nb[0] - 1, xa + (oxhi - ox));
                                    } else {
                                        xa = tx;
                                        xb = bx + oxhi;
                                    }
                                }
                                const unsigned hb = gballot<G>(gmask, gbase, have);
                                if (!hb) break;
                                int len = 0, j0r = 0;
                                if (have) {
                                    j0r = __ldg(&st.bstart[krow + xa]);
                                    len = __ldg(&st.bstart[krow + xb + 1]) - j0r;
                                }
                                int ltot;
                                const int lex = gexcl_scan<G>(gmask, len, gl, ltot);
                                // runs without particles take no entry: starts stay distinct
                                const bool ent = have && len > 0;
                                const unsigned hn = gballot<G>(gmask, gbase, ent);
                                const int slot = nrun + __popc(hn & ((1u << gl) - 1));
                                if (ent && slot < NRUN) {
                                    S.w.run.start[slot] = npart + lex;
                                    S.w.run.j0[slot] = j0r;
                                    // x offset of a particle = oxb + its block index
                                    S.w.run.oxb[slot] = (ox - xa) - krow;
                                    // offsets (oy, oz) and the run's image shift (m0, my, mz)
                                    S.w.run.oyz[slot] = (oy + 64) | ((oz + 64) << 8) | ((m0 + 8) << 16) | myz;
                                }
                                nrun += __popc(hn);
                                npart += ltot;
                                if (have) ox += xb - xa + 1;
                            }
                        }
                        if (nrun > NRUN) { give_up = true; break; }
                        __syncwarp(gmask);
                        // 2. all particles of all runs, G at a time
                        int rp = 0;  // the first run that starts at or after v0
#pragma unroll 1
                        for (int v0 = 0; v0 < npart; v0 += G) {
                            // the runs that start in this round, one per lane: a bit each
                            unsigned sb = 0;
                            if (rp + gl < nrun) {
                                const int s0 = S.w.run.start[rp + gl];
                                if (s0 < v0 + G) sb = 1u << (s0 - v0);
                            }
                            const unsigned smask = __reduce_or_sync(gmask, sb);
                            const int v = v0 + gl;
                            bool keep = false;
                            float qx = 0.f, qy = 0.f, qz = 0.f, qq = 0.f;
                            int j = 0, img = 0;
                            if (v < npart) {
                                // last run with start <= v
                                const int lo = rp + __popc(smask & (0xffffffffu >> (31 - gl))) - 1;
                                j = S.w.run.j0[lo] + (v - S.w.run.start[lo]);
                                const int oyz = S.w.run.oyz[lo];
                                const int oy = (oyz & 0xff) - 64, oz = ((oyz >> 8) & 0xff) - 64;
                                const int oxj = S.w.run.oxb[lo] + __ldg(&st.sblk[j]);
                                const float4 pj = __ldg(&st.p32[j]);
                                cand32(g, o0, o1, o2, pj, oxj, oy, oz, qx, qy, qz, qq);
                                keep = qq < rho2 && qq >= lo2 && !(j == i && oxj == 0 && oy == 0 && oz == 0);
                                img = pack_img(((oyz >> 16) & 15) - 8, ((oyz >> 20) & 15) - 8, ((oyz >> 24) & 15) - 8);
                            }
                            const unsigned bal = gballot<G>(gmask, gbase, keep);
                            const int pos = count + __popc(bal & ((1u << gl) - 1));
                            if (keep && pos < KMAX) {
                                S.x.pf.q[pos] = make_float4(qx, qy, qz, qq);
                                S.x.pf.r[pos] = make_int2(j, img);
                            }
                            count += __popc(bal);
                            rp += __popc(smask);
                        }
                        __syncwarp(gmask);
                        if (count <= KMAX) break;
                        rho *= 0.8f * cbrt_a((float)KMAX * rcp_a((float)count));
                    }
                    if (!give_up && count <= KMAX) {
                        // order by radial bucket: NBIN shells of equal volume inside
                        // rho (about equal counts; for a second round, of the shell
                        // above lo2 taken the same way); inside a bucket the gather
                        // order, which is deterministic, is kept
                        const float irho2 = rcp_a(rho2 - lo2);
                        int bin[KMAX / G];
#pragma unroll
                        for (int e2 = 0; e2 < KMAX / G; e2++) {
                            const int slot = e2 * G + gl;
                            bin[e2] = NBIN;
                            if (slot < count) {
                                const float t = fminf(fmaxf(S.x.pf.q[slot].w - lo2, 0.f) * irho2, 1.f);
                                bin[e2] = min(NBIN - 1, (int)((float)NBIN * t * sqrt_a(t)));
                            }
                        }
                        if constexpr (NBIN * (KMAX / G) == G) {
                            // counting sort by bin, stable in (row, lane) order: the
                            // count of every (bin, row) pair, one pair per lane, an
                            // exclusive scan over them in (bin, row) order, and each
                            // element's rank among its equals in its row
                            int *hist = S.w.run.start;  // the run table is free again
                            constexpr int ROWS = KMAX / G;
                            hist[gl] = 0;  // G entries: one per (bin, row) pair
                            __syncwarp(gmask);
                            int rank[ROWS];
#pragma unroll
                            for (int e2 = 0; e2 < ROWS; e2++) {
                                const unsigned eq = __match_any_sync(gmask, bin[e2]);
                                const unsigned eqg = G == 32 ? eq : (eq >> gbase);
                                rank[e2] = __popc(eqg & ((1u << gl) - 1));
                                // the lowest lane of each group of equals writes its count
                                if (bin[e2] < NBIN && rank[e2] == 0) hist[bin[e2] * ROWS + e2] = __popc(eqg);
                            }
                            __syncwarp(gmask);
                            const int mine = hist[gl];
                            int htot;
                            const int start = gexcl_scan<G>(gmask, mine, gl, htot);
                            __syncwarp(gmask);
                            hist[gl] = start;
                            __syncwarp(gmask);
#pragma unroll
                            for (int e2 = 0; e2 < ROWS; e2++)
                                if (bin[e2] < NBIN) S.x.pf.slot[hist[bin[e2] * ROWS + e2] + rank[e2]] = e2 * G + gl;
                        } else {
                            int pos0 = 0;
                            for (int b = 0; b < NBIN; b++) {
#pragma unroll
                                for (int e2 = 0; e2 < KMAX / G; e2++) {
                                    const unsigned m = gballot<G>(gmask, gbase, bin[e2] == b);
                                    if (bin[e2] == b) S.x.pf.slot[pos0 + __popc(m & ((1u << gl) - 1))] = e2 * G + gl;
                                    pos0 += __popc(m);
                                }
                            }
                        }
                        src.mode = 0;
                        src.count = count;
                        src.u = 0;
                        if (pp.collect && gl == 0) S.cnt[5] += count;
                        src.rho2 = rho2;
                        src.rg[0] = rg0; src.rg[1] = rg1; src.rg[2] = rg2;
                    } else if constexpr (HOT) {
                        // no preload list: the general kernel walks this cell
                        src.mode = 3;
                        flags |= 32;
                    }
                    __syncwarp(gmask);
                }
            }
            unsigned want = 0;
            T stop = stop2();

            for (int guard = 0; guard < (1 << 30); guard++) {
                // ---------------------------------- refill the candidate batch
                while (want == 0) {
                    const int mode = src.mode;
                    if (mode == 3) break;
                    if constexpr (F32) {
                        if (mdirty) {
                            // packed in (slot, lane) order, zeros up to the next
                            // multiple of 8
                            int mpos = 0;
#pragma unroll
                            for (int s = 0; s < VPL; s++) {
                                const unsigned oc = gballot<G>(gmask, gbase, tri[s] != TRI_EMPTY);
                                if (tri[s] != TRI_EMPTY)
                                    S.v4[mpos + __popc(oc & ((1u << gl) - 1))] = make_float4(vx[s], vy[s], vz[s], kap[s]);
                                mpos += __popc(oc);
                            }
                            if (gl < ((ntri + 7) & ~7) - ntri) S.v4[ntri + gl] = make_float4(0.f, 0.f, 0.f, 0.f);
                            mdirty = false;
                            __syncwarp(gmask);
                        }
                    }
                    if (mode == 0) {
                        const int u = src.u, count = src.count;
                        if (u >= count) {
                            if ((T)stop <= (T)src.rho2 * (T)0.9999) {
                                src.mode = 3;
                            } else if constexpr (HOT) {
                                // the bound reaches past the preload: once a wider
                                // preload, then the general kernel
                                src.mode = 3;
                                if (src.round == 0) {
                                    __syncwarp(gmask);
                                    src.round = 1;
                                    src.fell_back = 2;  // a shortfall, met by a second preload
                                    src.lo2 = src.rho2;
                                    __syncwarp(gmask);
                                    goto regather;
                                }
                                flags |= 32;
                            } else {
                                src.mode = 1;
                                src.fell_back = 1;
                            }
                            continue;
                        }
                        const int idx = u + gl;
                        const bool in = idx < count;
                        // the first batch meets the initial box: nothing to drop yet
                        const int nb0 = src.nbatch;
                        const bool filt = nb0 > 0;
                        bool ok = false;
                        T cqq = 0;
                        __syncwarp(gmask);  // the previous batch has been read
                        if (in) {
                            const int slot = S.x.pf.slot[idx];
                            const float4 q4 = S.x.pf.q[slot];
                            const int2 r = S.x.pf.r[slot];
                            cqq = (T)q4.w;
                            const T crj = st.radical ? (T)__ldg(&st.p32[r.x]).w : (T)0;
                            S.cbq[gl] = mk4<T>((T)q4.x, (T)q4.y, (T)q4.z, (T)q4.w);
                            S.cbr[gl] = r;
                            S.cbrj[gl] = crj;
                            ok = (T)q4.w < stop;
                            if constexpr (F32) {
                                if (filt && ok && q4.w >= 1e-30f) {
                                    const float cc = st.radical ? 0.5f * (q4.w + rp32 * rp32 - crj * crj) : 0.5f * q4.w;
                                    ok = may_cut(S.v4, ((ntri + 7) & ~7), q4.x, q4.y, q4.z, cc,
                                                 VG_RARE(q4.w < qabs2) ? band_close(tol32f, r2, q4.w, eabs)
                                                                       : tol32f * sqrt_a(r2 * q4.w));
                                }
                            }
                        }
                        want = gballot<G>(gmask, gbase, ok);
                        __syncwarp(gmask);
                        src.nbatch = nb0 + 1;  // every gl writes the same value
                        // bucketed: once the last entry's bucket starts beyond the
                        // bound, every later entry lies beyond it too
                        const int last = min(count - u, G) - 1;
                        const float qlast = __shfl_sync(gmask, (float)cqq, last, G);  // this batch's gl value
                        const float plo2 = src.lo2, pw2 = src.rho2 - plo2;
                        const float t = fminf(fmaxf(qlast - plo2, 0.f) * rcp_a(pw2), 1.f);
                        const int bl = min(NBIN - 1, (int)((float)NBIN * t * sqrt_a(t)));
                        // bucket bl starts at t = (bl / NBIN)^(2/3)
                        const float lb2 = (plo2 + pw2 * bucket_t[bl]) * 0.9999f;  // margin for rounding
                        src.u = ((T)lb2 >= stop) ? count : u + G;
                        continue;
                    }
                    if constexpr (HOT) {
                        break;  // modes 1 and 2 (the walk) never occur here
                    } else {
                    const int vp = src.vp, vtot = src.vtot;
                    if (vp < vtot) {
                        // a batch of the current window's particles
                        const int v = vp + gl;
                        const int nb0 = src.nbatch;
                        const bool filt = nb0 > 0;
                        bool ok = false;
                        __syncwarp(gmask);  // the previous batch has been read
                        if (v < vtot) {
                            T cqx = 0, cqy = 0, cqz = 0, cqq = 0, crj = 0;
                            int lo = 0, hi = src.nwin - 1;  // last block with vstart <= v
                            while (lo < hi) {
                                const int mid = (lo + hi + 1) >> 1;
                                if (S.w.win.vstart[mid] <= v) lo = mid; else hi = mid - 1;
                            }
                            const int j = S.w.win.j0[lo] + (v - S.w.win.vstart[lo]);
                            const int oc = S.w.win.o[lo], mc = S.w.win.m[lo];
                            const int ox = imgc(oc, 0), oy = imgc(oc, 1), oz = imgc(oc, 2);
                            if constexpr (F32) {
                                const float4 pj = __ldg(&st.p32[j]);
                                float qx, qy, qz, qq;
                                cand32(g, o0, o1, o2, pj, ox, oy, oz, qx, qy, qz, qq);
                                cqx = qx; cqy = qy; cqz = qz; cqq = qq; crj = pj.w;
                                // bit 24 of the packed offset: inside the prefetch box
                                ok = !(((oc >> 24) & 1) && qq < src.rho2);
                            } else {
                                const D4 pj = st.p64[j];
                                cand64(g, S.cc, pj, imgc(mc, 0), imgc(mc, 1), imgc(mc, 2), cqx, cqy, cqz, cqq);
                                crj = pj.w;
                                ok = true;
                            }
                            if (ox == 0 && oy == 0 && oz == 0 && j == i) ok = false;
                            ok = ok && cqq < stop;
                            if constexpr (F32) {
                                if (filt && ok && cqq >= 1e-30f) {
                                    const float cc = st.radical ? 0.5f * (cqq + rp32 * rp32 - crj * crj) : 0.5f * cqq;
                                    ok = may_cut(S.v4, ((ntri + 7) & ~7), cqx, cqy, cqz, cc,
                                                 VG_RARE(cqq < qabs2) ? band_close(tol32f, r2, cqq, eabs)
                                                                      : tol32f * sqrt_a(r2 * cqq));
                                }
                            }
                            S.cbq[gl] = mk4<T>(cqx, cqy, cqz, cqq);
                            S.cbr[gl] = make_int2(j, mc & 0xffffff);
                            S.cbrj[gl] = crj;
                        }
                        want = gballot<G>(gmask, gbase, ok);
                        __syncwarp(gmask);
                        src.nbatch = nb0 + 1;  // every gl writes the same value
                        src.vp = vp + G;
                        continue;
                    }
                    // a new window: up to G blocks set up in parallel
                    if (src.last) { src.mode = 3; continue; }
                    int ox = 0, oy = 0, oz = 0, nsidx = 0;
                    bool cand = false;
                    if (mode == 1) {
                        const int e = src.e;
                        const int ocount = SY.off_count, obase = SY.off_base;
                        if (e >= ocount) { src.mode = 2; continue; }
                        const int ei = e + gl;
                        bool beyond = true;
                        if (ei < ocount) {
                            const float lb = __ldg(&off.lb[obase + ei]);
                            beyond = (T)(lb * lb) * (T)0.99998 >= stop;
                            const int code = __ldg(&off.code[obase + ei]);
                            ox = imgc(code, 0); oy = imgc(code, 1); oz = imgc(code, 2);
                        }
                        // the list is sorted by its bound: entries past the first
                        // one beyond the stop radius are all beyond it
                        const unsigned bb = gballot<G>(gmask, gbase, beyond);
                        const int first = bb ? __ffs(bb) - 1 : G;
                        cand = gl < first;
                        if (first < G && e + first < ocount) src.last = 1;
                        src.e = e + G;
                    } else {
                        const int shell = src.shell;
                        const float hmin = fminf(g.hf[0], fminf(g.hf[1], g.hf[2]));
                        const float sb = (float)(shell - 1) * hmin;
                        if ((T)(sb * sb) * (T)0.99998 >= stop) { src.mode = 3; continue; }
                        // shells up to 640 keep (2 shell + 1)^3 within 32-bit indices
                        const int maxs = min(640, SY.off_shell + MAX_SHELL_EXTRA + 2 * max(g.nb[0], max(g.nb[1], g.nb[2])));
                        if (shell > maxs) { src.limit = 1; src.mode = 3; continue; }
                        // the shell's surface only: two z faces (wd^2 each), two y faces
                        // (wd (wd - 2)), two x faces ((wd - 2)^2)
                        const int wd = 2 * shell + 1, sidx = src.sidx;
                        const int fa = wd * wd, fb = wd * (wd - 2), fc = (wd - 2) * (wd - 2);
                        if (sidx >= 2 * (fa + fb + fc)) { src.shell = shell + 1; src.sidx = 0; continue; }
                        const int si = sidx + gl;
                        if (si < 2 * (fa + fb + fc)) {
                            shell_member(si, shell, ox, oy, oz);
                            const float lbmax = (float)SY.off_shell * hmin;
                            const float lbx = fmaxf(0.f, (float)(abs(ox) - 1)) * g.hf[0];
                            const float lby = fmaxf(0.f, (float)(abs(oy) - 1)) * g.hf[1];
                            const float lbz = fmaxf(0.f, (float)(abs(oz) - 1)) * g.hf[2];
                            // shell members that the offset list did not hold
                            cand = !(lbx * lbx + lby * lby + lbz * lbz < lbmax * lbmax);
                        }
                        // the cursor moves after the window's ballot, once every
                        // lane has read it
                        nsidx = sidx + G;
                    }
                    int kk = 0, mx = 0, my = 0, mz = 0, len = 0, j0b = 0, inpref = 0;
                    if (cand) {
                        cand = resolve(g, SY.blk_base, S.cc.b, ox, oy, oz, kk, mx, my, mz);
                        if (cand) {
                            const float gap2 = block_gap2(g, o0, o1, o2, ox, oy, oz);
                            cand = !((T)gap2 * (T)0.99998 >= stop);
                        }
                        if (cand) {
                            j0b = __ldg(&st.bstart[kk]);
                            len = __ldg(&st.bstart[kk + 1]) - j0b;
                            cand = len > 0;
                            if constexpr (F32) {
                                // beyond the offset list (extended cells): the block bound, for
                                // blocks whose particles would cost more than the test
                                if (cand && mode == 2 && len >= 8) {
                                    const float bl0 = (float)ox * g.hf[0] - o0, bl1 = (float)oy * g.hf[1] - o1,
                                                bl2 = (float)oz * g.hf[2] - o2;
                                    const float ex = st.radical ? (float)(S.cc.rmax * S.cc.rmax - S.cc.rp * S.cc.rp) : 0.f;
                                    const float sl = 1e-5f * (sqrt_a((float)r2) + fmaxf(g.hf[0], fmaxf(g.hf[1], g.hf[2])));
                                    cand = block_touches(S.v4, ((ntri + 7) & ~7), bl0, bl1, bl2, bl0 + g.hf[0],
                                                         bl1 + g.hf[1], bl2 + g.hf[2], fmaxf(ex, 0.f), sl);
                                }
                            }
                            // particles the prefetch already offered: inside its
                            // block box, in a row it gathered, closer than its radius
                            const float rho2 = src.rho2;
                            inpref = rho2 > 0.f && abs(ox) <= src.rg[0] && abs(oy) <= src.rg[1] &&
                                     abs(oz) <= src.rg[2] && row_gap2(g, o1, o2, oy, oz) < rho2 &&
                                     block_gap2(g, o0, o1, o2, ox, oy, oz) < rho2;
                        }
                    }
                    const unsigned cb = gballot<G>(gmask, gbase, cand);
                    int ltot;
                    const int lex = gexcl_scan<G>(gmask, cand ? len : 0, gl, ltot);
                    if (cand) {
                        const int slot = __popc(cb & ((1u << gl) - 1));
                        S.w.win.vstart[slot] = lex;
                        S.w.win.j0[slot] = j0b;
                        S.w.win.o[slot] = pack_img(ox, oy, oz) | (inpref << 24);
                        S.w.win.m[slot] = pack_img(mx, my, mz);
                    }
                    if (mode == 2) src.sidx = nsidx;
                    src.nwin = __popc(cb);
                    src.vp = 0;
                    src.vtot = ltot;
                    __syncwarp(gmask);
                    }  // !HOT
                }
                if (want == 0) break;
                const int srcl = __ffs(want) - 1;
                want &= want - 1;
                const auto cq4 = S.cbq[srcl];
                const int2 cr = S.cbr[srcl];
                const T qx = cq4.x, qy = cq4.y, qz = cq4.z, qq = cq4.w;
                const int ref = cr.x, img = cr.y;
                if (qq >= stop) continue;
                if (VG_RARE(qq < (T)1e-30)) {
                    // coincident: in FP32 perhaps only after rounding, so a retry
                    if constexpr (F32) { flags |= 2; break; }
                    flags |= 8;
                    continue;
                }
                T c;
                if (st.radical) {
                    const T rj = S.cbrj[srcl];
                    if constexpr (F32) c = 0.5f * (qq + rp32 * rp32 - rj * rj);
                    else c = 0.5 * (qq + S.cc.rp * S.cc.rp - rj * rj);
                } else {
                    c = (T)0.5 * qq;
                }

                // ================================= cut by the plane q.r = c
                if (VG_RARE(pp.collect) && gl == 0) { S.cnt[0]++; S.cnt[1] += ntri; }
                unsigned outm = 0, nearm = 0, onm = 0;
                if constexpr (F32) {
                    // |d| against the band tau * kappa, squared (no square root on
                    // the critical path): out if d > band, near if |d| <= band
                    float t2 = tol32f * tol32f * r2 * qq;
                    if (VG_RARE(qq < qabs2)) {
                        const float b = band_close(tol32f, r2, qq, eabs);
                        t2 = b * b;
                    }
#pragma unroll
                    for (int s = 0; s < VPL; s++) {
                        if ((rows >> s) & 1) {
                            const float d = vx[s] * qx + vy[s] * qy + vz[s] * qz - c;
                            const float b2 = t2 * (kap[s] * kap[s]);
                            if (tri[s] != TRI_EMPTY) {
                                if (d > 0.f && d * d > b2) outm |= 1u << s;
                                else if (d * d <= b2) nearm |= 1u << s;
                            }
                        }
                    }
                } else {
                    const T tau = (T)(pp.tau_rel * g.s * sqrt((double)qq));
#pragma unroll
                    for (int s = 0; s < VPL; s++) {
                        if ((rows >> s) & 1) {
                            const T d = vx[s] * qx + vy[s] * qy + vz[s] * qz - c;
                            if (tri[s] != TRI_EMPTY) {
                                if (d > tau) outm |= 1u << s;
                                else if (d >= -tau) onm |= 1u << s;
                            }
                        }
                    }
                }
                if constexpr (F32) {
                    if (VG_RARE(__any_sync(gmask, nearm))) {
                        if (pp.collect && gl == 0) S.cnt[4]++;
#pragma unroll
                        for (int s = 0; s < VPL; s++) {
                            if (nearm & (1u << s)) {
                                const int r = classify64(&g, &st, &S.cc, S.pref, S.pimg, tri[s], ref, img,
                                                         pp.tau_rel * g.s);
                                if (r > 0) outm |= 1u << s;
                                else if (r == 0) onm |= 1u << s;
                            }
                        }
                    }
                }
                if (!__any_sync(gmask, outm)) continue;
                if (__any_sync(gmask, onm)) flags |= 1;
                if (F32 && VG_RARE((float)qq < qclose2)) flags |= 16;
                if (VG_RARE(pp.collect) && gl == 0) S.cnt[2]++;
                int np = -1;
                if (nplane < MAXP) {
                    np = nplane++;
                } else if constexpr (HOT) {
                    flags |= 32;  // plane slots used up: the general kernel
                    break;
                } else {
                    live_planes();
#pragma unroll
                    for (int w2 = NW - 1; w2 >= 0; w2--)
                        if (~live[w2]) np = w2 * 64 + __ffsll((long long)~live[w2]) - 1;
                }
                if (VG_RARE(np < 0)) { flags |= 2; break; }
                // the removed triangles: R of them, numbered in (slot, lane) order
                const unsigned lt = (1u << gl) - 1;
                int R = 0, rpos[VPL];
#pragma unroll
                for (int s = 0; s < VPL; s++) {
                    const unsigned m = gballot<G>(gmask, gbase, (outm >> s) & 1);
                    rpos[s] = R + __popc(m & lt);
                    R += __popc(m);
                }
                const int K = ntri - R;  // kept vertices
                int N = 0;
                if (R * 3 <= G) {
                    // every directed edge of a removed triangle in a lane of its own;
                    // an edge (x,y) borders the kept part iff its twin (y,x) was not
                    // removed, and the twin carries the same unordered pair: a match
                    // over the group finds it
#pragma unroll
                    for (int s = 0; s < VPL; s++) {
                        if (outm & (1u << s)) {
                            const int a = tri_a(tri[s]), b = tri_b(tri[s]), cc = tri_c(tri[s]);
                            S.elist[3 * rpos[s]] = a | (b << 8);
                            S.elist[3 * rpos[s] + 1] = b | (cc << 8);
                            S.elist[3 * rpos[s] + 2] = cc | (a << 8);
                        }
                    }
                    __syncwarp(gmask);
                    const bool have = gl < 3 * R;
                    const int e = have ? S.elist[gl] : 0;
                    const int ex = e & 0xff, ey = e >> 8;
                    // idle lanes share one key: the match's cost grows with
                    // the number of distinct keys
                    const unsigned key = have ? (unsigned)(min(ex, ey) | (max(ex, ey) << 8)) : 0xffffffffu;
                    // every lane of the group takes part in the match (not behind &&)
                    const unsigned same = __match_any_sync(gmask, key);
                    const bool bd = have && __popc(same) == 1;
                    const unsigned bm = gballot<G>(gmask, gbase, bd);
                    N = __popc(bm);
                    __syncwarp(gmask);  // every lane has read its edge
                    if (bd) S.elist[__popc(bm & lt)] = e;
                } else {
                    // many removed: mark their directed edges in the bit matrix
#pragma unroll
                    for (int s = 0; s < VPL; s++) {
                        if (outm & (1u << s)) {
                            const int a = tri_a(tri[s]), b = tri_b(tri[s]), cc = tri_c(tri[s]);
                            atomicOr(&S.E[a][b >> 5], 1u << (b & 31));
                            atomicOr(&S.E[b][cc >> 5], 1u << (cc & 31));
                            atomicOr(&S.E[cc][a >> 5], 1u << (a & 31));
                        }
                    }
                    __syncwarp(gmask);
                    unsigned bnd[VPL];
                    int nc = 0;
#pragma unroll
                    for (int s = 0; s < VPL; s++) {
                        bnd[s] = 0;
                        if (outm & (1u << s)) {
                            const int a = tri_a(tri[s]), b = tri_b(tri[s]), cc = tri_c(tri[s]);
                            if (!((S.E[b][a >> 5] >> (a & 31)) & 1)) bnd[s] |= 1;
                            if (!((S.E[cc][b >> 5] >> (b & 31)) & 1)) bnd[s] |= 2;
                            if (!((S.E[a][cc >> 5] >> (cc & 31)) & 1)) bnd[s] |= 4;
                            nc += __popc(bnd[s]);
                        }
                    }
                    __syncwarp(gmask);
                    // every gl has read the matrix: each clears the words it set
#pragma unroll
                    for (int s = 0; s < VPL; s++) {
                        if (outm & (1u << s)) {
                            const int a = tri_a(tri[s]), b = tri_b(tri[s]), cc = tri_c(tri[s]);
                            S.E[a][b >> 5] = 0u;
                            S.E[b][cc >> 5] = 0u;
                            S.E[cc][a >> 5] = 0u;
                        }
                    }
                    int npos;
                    if constexpr (VPL <= 4) {
                        // exclusive prefix by bit planes: independent ballots
                        // instead of a chain of shuffles
                        npos = 0;
#pragma unroll
                        for (int b = 0; (1 << b) <= 3 * VPL; b++) {
                            const unsigned m = gballot<G>(gmask, gbase, (nc >> b) & 1);
                            npos += __popc(m & lt) << b;
                            N += __popc(m) << b;
                        }
                    } else {
                        npos = gexcl_scan<G>(gmask, nc, gl, N);
                    }
                    if (K + N <= CAP) {
#pragma unroll
                        for (int s = 0; s < VPL; s++) {
                            if (outm & (1u << s)) {
                                const int a = tri_a(tri[s]), b = tri_b(tri[s]), cc = tri_c(tri[s]);
                                if (bnd[s] & 1) S.elist[npos++] = a | (b << 8);
                                if (bnd[s] & 2) S.elist[npos++] = b | (cc << 8);
                                if (bnd[s] & 4) S.elist[npos++] = cc | (a << 8);
                            }
                        }
                    }
                }
                const int tot = K + N;
                if (VG_RARE(pp.collect) && gl == 0) S.cnt[3] += N;
                const int rc = tot > CAP ? 3 : (tot == 0 ? 2 : 1);
                if (VG_RARE(rc != 1)) {
                    // no vertex left: an empty power cell, but for a Voronoi
                    // cell (which holds its particle) a numerical failure
                    flags |= (rc == 2 && st.radical) ? 4 : 2;
                    break;
                }
#pragma unroll
                for (int s = 0; s < VPL; s++)
                    if (outm & (1u << s)) tri[s] = TRI_EMPTY;  // removed: its slot is free
                if (gl == 0) {
                    S.pl[np] = mk4<T>(qx, qy, qz, c);
                    S.pref[np] = ref;
                    S.pimg[np] = img;
                }
                __syncwarp(gmask);
                // kept vertices stay in place; free slots take the new ones in
                // order, each solving its own from the boundary edge list
                ntri = tot;
                unsigned need = 0;
                int rk[VPL];
                {
                    int rank0 = 0;
#pragma unroll
                    for (int s = 0; s < VPL; s++) {
                        const bool fr = tri[s] == TRI_EMPTY;
                        const unsigned fm = gballot<G>(gmask, gbase, fr);
                        rk[s] = rank0 + __popc(fm & lt);
                        rank0 += __popc(fm);
                        if (fr && rk[s] < N) need |= 1u << s;
                    }
                }
                // a new vertex: planes x, y and the cutting plane; a lane with two
                // slots to fill takes a second round
#pragma unroll 1
                while (__any_sync(gmask, need)) {
                    if (need) {
                        const int s0 = __ffs(need) - 1;
                        int q = rk[0];
#pragma unroll
                        for (int s = 1; s < VPL; s++)
                            if (s == s0) q = rk[s];
                        const int xy = S.elist[q];
                        const int x = xy & 0xff, y = xy >> 8;
                        const auto P1 = S.pl[x];
                        const auto P2 = S.pl[y];
                        const T x23x = P2.y * qz - P2.z * qy, x23y = P2.z * qx - P2.x * qz, x23z = P2.x * qy - P2.y * qx;
                        const T x31x = qy * P1.z - qz * P1.y, x31y = qz * P1.x - qx * P1.z, x31z = qx * P1.y - qy * P1.x;
                        const T x12x = P1.y * P2.z - P1.z * P2.y, x12y = P1.z * P2.x - P1.x * P2.z,
                                x12z = P1.x * P2.y - P1.y * P2.x;
                        const T det = P1.x * x23x + P1.y * x23y + P1.z * x23z;
                        T nx, ny, nz;
                        float kp = 1.f, m123 = 0.f;
                        bool solved = false;
                        if constexpr (F32) {
                            m123 = (P1.x * P1.x + P1.y * P1.y + P1.z * P1.z) *
                                   (P2.x * P2.x + P2.y * P2.y + P2.z * P2.z) * qq;
                            const float d2 = det * det;
                            if (VG_RARE(!(d2 * KAP_MAX2 >= m123))) {
                                const float3 v = solve_new64(&g, &st, &S.cc, S.pref, S.pimg, x, y, ref, img);
                                nx = v.x; ny = v.y; nz = v.z;
                                solved = true;
                            }
                        }
                        if (!solved) {
                            T id;
                            if constexpr (F32) {
                                id = rcp_a(det);
                                kp = fmaxf(1.f, sqrt_a(m123) * fabsf(id) * (1.f / KAP0));
                            } else {
                                id = (T)1 / det;
                            }
                            nx = (P1.w * x23x + P2.w * x31x + c * x12x) * id;
                            ny = (P1.w * x23y + P2.w * x31y + c * x12y) * id;
                            nz = (P1.w * x23z + P2.w * x31z + c * x12z) * id;
                        }
                        const unsigned tn = mk_tri(x, y, np);
#pragma unroll
                        for (int s = 0; s < VPL; s++) {
                            if (s == s0) {
                                tri[s] = tn;
                                vx[s] = nx; vy[s] = ny; vz[s] = nz;
                                kap[s] = kp;
                            }
                        }
                        need &= need - 1;
                    }
                }
                T rr = 0;
                rows = 0;
                // every vertex lies on an old edge, so within the old radius: one
                // beyond it, or not finite, is a numerical failure (rr = inf
                // carries it through the group maximum to every lane)
                const T r2lim = r2 * (T)1.01;
                bool wild = false;
#pragma unroll
                for (int s = 0; s < VPL; s++) {
                    if (tri[s] != TRI_EMPTY) {
                        T q2 = vx[s] * vx[s] + vy[s] * vy[s] + vz[s] * vz[s];
                        wild |= !(q2 <= r2lim);
                        if constexpr (F32) q2 *= 1.f + 4e-6f * kap[s];  // allowance for FP32 error
                        rr = rr > q2 ? rr : q2;
                    }
                    if (__any_sync(gmask, tri[s] != TRI_EMPTY)) rows |= 1u << s;
                }
                if constexpr (F32) mdirty = true;
                if (VG_RARE(wild)) rr = (T)INFINITY;
                r2 = gmax<G>(gmask, rr);
                if (VG_RARE(!(r2 < (T)INFINITY))) { flags |= 2; break; }
                __syncwarp(gmask);
                stop = stop2();
            }

            // ================================================= statistics
            live_planes();
            bool degen = flags & (1 | 16);
            if constexpr (F32) {
                // an ill-conditioned vertex (kappa >= 64) is off by more than
                // the 1e-5 bar allows: the statistics take FP64 vertices
                bool hk = false;
#pragma unroll
                for (int s = 0; s < VPL; s++) hk |= tri[s] != TRI_EMPTY && kap[s] >= 64.f;
                const bool anyhk = __any_sync(gmask, hk);
                degen = degen || anyhk;
            }
            if constexpr (HOT) {
                // FP64 statistics, the walk or a second round of faces needed:
                // the general kernel computes the cell (flags are warp-uniform)
                int nlive = 0;
#pragma unroll
                for (int w2 = 0; w2 < NW; w2++) nlive += __popcll(live[w2]);
                if (degen || (flags & 32) || nlive > G) {
                    if (gl == 0) {
                        const int slot = atomicAdd(o.retry0_count, 1);
                        o.retry0[slot] = i;
                    }
                    __syncwarp(gmask);
                    continue;
                }
            }
            bool fail = flags & 2;
            int status = VG_CELL_OK;
            if (flags & 4) status = VG_CELL_EMPTY;
            else if (flags & 8) status = VG_CELL_DUP;
            else if (src.limit) status = VG_CELL_LIMIT;
            const int out_i = S.cc.self_id;
            if (!fail && status == VG_CELL_OK) {
                const int T_ = ntri;
#pragma unroll
                for (int s = 0; s < VPL; s++) {
                    const int t = s * G + gl;
                    S.x.v.stri[t] = tri[s]; S.x.v.sx[t] = vx[s]; S.x.v.sy[t] = vy[s]; S.x.v.sz[t] = vz[s];
                }
                // reference point for the fans: a vertex of the cell (a radical
                // cell may lie far from its particle, where fans from the
                // particle would cancel)
                int tref = 0;
                T rx = 0, ry = 0, rz = 0;
                {
                    int rsl = 0;
                    unsigned occ = gballot<G>(gmask, gbase, tri[0] != TRI_EMPTY);
#pragma unroll
                    for (int s = 1; s < VPL; s++) {
                        const unsigned oc = gballot<G>(gmask, gbase, tri[s] != TRI_EMPTY);
                        if (!occ && oc) { occ = oc; rsl = s; }
                    }
                    const int rl = __ffs(occ) - 1;
                    tref = rsl * G + rl;
                    T cxv = 0, cyv = 0, czv = 0;
#pragma unroll
                    for (int s = 0; s < VPL; s++)
                        if (s == rsl) { cxv = vx[s]; cyv = vy[s]; czv = vz[s]; }
                    rx = __shfl_sync(gmask, cxv, rl, G);
                    ry = __shfl_sync(gmask, cyv, rl, G);
                    rz = __shfl_sync(gmask, czv, rl, G);
                }
                // pass 0 sums the FP32 vertices; a cell thin against its
                // distance from the particle gets a pass from FP64 vertices
                for (int pass = 0; pass < 2; pass++) {
                if (!HOT && degen) {
                    // (vertices read back from the staging arrays: the loop stays rolled)
#pragma unroll 1
                    for (int s = 0; s < VPL; s++) {
                        const int t = s * G + gl;
                        const unsigned tr = S.x.v.stri[t];
                        if (tr != TRI_EMPTY) {
                            if constexpr (F32) {
                                vertex64(&g, &st, &S.cc, S.pref, S.pimg, tr, S.x.v.dpos[t]);
                            } else {
                                S.x.v.dpos[t][0] = S.x.v.sx[t]; S.x.v.dpos[t][1] = S.x.v.sy[t]; S.x.v.dpos[t][2] = S.x.v.sz[t];
                            }
                        }
                    }
                }
                __syncwarp(gmask);
                double dref[3];
                if (!HOT && degen) { dref[0] = S.x.v.dpos[tref][0]; dref[1] = S.x.v.dpos[tref][1]; dref[2] = S.x.v.dpos[tref][2]; }
                else { dref[0] = (double)rx; dref[1] = (double)ry; dref[2] = (double)rz; }
                int F = 0;
#pragma unroll
                for (int w2 = 0; w2 < NW; w2++) F += __popcll(live[w2]);
                double vol = 0.0;  // six times the volume, accumulated in FP64
                T cx = 0, cy = 0, cz = 0, area = 0;
                int order_sum = 0, faces_kept = 0;
                bool bad = false;
                unsigned long long key[R];
#pragma unroll
                for (int r = 0; r < R; r++) key[r] = ~0ull;
#pragma unroll 1
                for (int rnd = 0; rnd * G < F; rnd++) {
                    const int f = rnd * G + gl;
                    // plane of face f: the f-th set bit of the live mask
                    int a = -1;
                    if (f < F) {
                        int cntw = 0;
#pragma unroll
                        for (int w2 = 0; w2 < NW; w2++) {
                            const int pc = __popcll(live[w2]);
                            if (a < 0 && f < cntw + pc) {
                                const unsigned lo32 = (unsigned)live[w2], hi32 = (unsigned)(live[w2] >> 32);
                                const int nth = f - cntw, plo = __popc(lo32);
                                a = w2 * 64 + (nth < plo ? (int)__fns(lo32, 0, nth + 1)
                                                         : 32 + (int)__fns(hi32, 0, nth - plo + 1));
                            }
                            cntw += pc;
                        }
                    }
                    // the neighbour's input index, asked for before the walk so that
                    // the load's round trip overlaps it
                    int nid_pre = 0;
                    if (a >= 0) {
                        const int ref0 = S.pref[a];
                        nid_pre = ref0 >= 0 ? __ldg(&st.sid[ref0]) : ref0;
                    }
                    // every vertex enters itself in the walk tables of its faces
#pragma unroll 1
                    for (int s = 0; s < VPL; s++) {
                        const int t = s * G + gl;
                        const unsigned tr = S.x.v.stri[t];
                        if (tr != TRI_EMPTY) {
                            const int pp3[3] = {tri_a(tr), tri_b(tr), tri_c(tr)};
#pragma unroll
                            for (int k3 = 0; k3 < 3; k3++) {
                                const int pl_ = pp3[k3], xx = pp3[(k3 + 1) % 3];
                                int rk = 0;
#pragma unroll
                                for (int w2 = 0; w2 < NW; w2++) {
                                    const int lo64 = w2 * 64;
                                    if (pl_ >= lo64 + 64) rk += __popcll(live[w2]);
                                    else if (pl_ > lo64) rk += __popcll(live[w2] & ((1ull << (pl_ - lo64)) - 1));
                                }
                                if (rk / G == rnd) {
                                    S.x.v.ftab[rk % G][xx] = (typename S_t::FT)t;
                                    S.sfirst[rk % G] = (typename S_t::FT)t;
                                }
                            }
                        }
                    }
                    __syncwarp(gmask);
                    const int t0 = a >= 0 ? (int)S.sfirst[gl] : -1;
                    if (a >= 0) {
                        int steps = 0, cur = t0;
                        bool closed = false;
                        int order = 0;
                        bool keep = true;
                        T farea;
                        if (HOT || !degen) {
                            const T u0x = S.x.v.sx[t0] - rx, u0y = S.x.v.sy[t0] - ry, u0z = S.x.v.sz[t0] - rz;
                            T fv = 0, fcx = 0, fcy = 0, fcz = 0, fax = 0, fay = 0, faz = 0;
#pragma unroll 1
                            for (steps = 0; steps < CAP; steps++) {
                                const unsigned tr = S.x.v.stri[cur];
                                const int p0 = tri_a(tr), p1 = tri_b(tr), p2 = tri_c(tr);
                                const int yy = p0 == a ? p2 : (p1 == a ? p0 : (p2 == a ? p1 : -1));
                                if (yy < 0) { bad = true; break; }
                                const int nx = S.x.v.ftab[gl][yy];
                                if (nx >= CAP || S.x.v.stri[nx] == TRI_EMPTY) { bad = true; break; }
                                if (nx == t0) { steps++; closed = true; break; }
                                if (cur != t0) {
                                    const T ax = S.x.v.sx[cur] - rx, ay = S.x.v.sy[cur] - ry, az = S.x.v.sz[cur] - rz;
                                    const T bx = S.x.v.sx[nx] - rx, by = S.x.v.sy[nx] - ry, bz = S.x.v.sz[nx] - rz;
                                    const T det = u0x * (ay * bz - az * by) - u0y * (ax * bz - az * bx) +
                                                  u0z * (ax * by - ay * bx);
                                    fv += det;
                                    fcx += det * (u0x + ax + bx);
                                    fcy += det * (u0y + ay + by);
                                    fcz += det * (u0z + az + bz);
                                    const T e1x = ax - u0x, e1y = ay - u0y, e1z = az - u0z;
                                    const T e2x = bx - u0x, e2y = by - u0y, e2z = bz - u0z;
                                    fax += e1y * e2z - e1z * e2y;
                                    fay += e1z * e2x - e1x * e2z;
                                    faz += e1x * e2y - e1y * e2x;
                                }
                                cur = nx;
                            }
                            vol += (double)fv;
                            cx += fcx; cy += fcy; cz += fcz;
                            if constexpr (F32) farea = 0.5f * sqrt_a(fax * fax + fay * fay + faz * faz);
                            else farea = (T)0.5 * sqrt(fax * fax + fay * fay + faz * faz);
                            order = steps;
                        } else {
                            // degenerate cell: FP64 vertices, coincident ones merged
                            const double eps = pp.merge_rel * g.s, eps2 = eps * eps;
                            const double fx = S.x.v.dpos[t0][0] - dref[0], fy = S.x.v.dpos[t0][1] - dref[1],
                                         fz = S.x.v.dpos[t0][2] - dref[2];
                            double px = fx, py = fy, pz = fz, per = 0, fv = 0, fcx = 0, fcy = 0, fcz = 0;
                            double fax = 0, fay = 0, faz = 0;
                            int distinct = 1;
#pragma unroll 1
                            for (steps = 0; steps < CAP; steps++) {
                                const unsigned tr = S.x.v.stri[cur];
                                const int p0 = tri_a(tr), p1 = tri_b(tr), p2 = tri_c(tr);
                                const int yy = p0 == a ? p2 : (p1 == a ? p0 : (p2 == a ? p1 : -1));
                                if (yy < 0) { bad = true; break; }
                                const int nx = S.x.v.ftab[gl][yy];
                                if (nx >= CAP || S.x.v.stri[nx] == TRI_EMPTY) { bad = true; break; }
                                if (nx == t0) { steps++; closed = true; break; }
                                const double A[3] = {S.x.v.dpos[cur][0] - dref[0], S.x.v.dpos[cur][1] - dref[1],
                                                     S.x.v.dpos[cur][2] - dref[2]};
                                const double B[3] = {S.x.v.dpos[nx][0] - dref[0], S.x.v.dpos[nx][1] - dref[1],
                                                     S.x.v.dpos[nx][2] - dref[2]};
                                if (cur != t0) {
                                    const double det = fx * (A[1] * B[2] - A[2] * B[1]) - fy * (A[0] * B[2] - A[2] * B[0]) +
                                                       fz * (A[0] * B[1] - A[1] * B[0]);
                                    fv += det;
                                    fcx += det * (fx + A[0] + B[0]);
                                    fcy += det * (fy + A[1] + B[1]);
                                    fcz += det * (fz + A[2] + B[2]);
                                    const double e1x = A[0] - fx, e1y = A[1] - fy, e1z = A[2] - fz;
                                    const double e2x = B[0] - fx, e2y = B[1] - fy, e2z = B[2] - fz;
                                    fax += e1y * e2z - e1z * e2y;
                                    fay += e1z * e2x - e1x * e2z;
                                    faz += e1x * e2y - e1y * e2x;
                                }
                                const double dx = B[0] - px, dy = B[1] - py, dz = B[2] - pz;
                                if (dx * dx + dy * dy + dz * dz > eps2) {
                                    per += sqrt(dx * dx + dy * dy + dz * dz);
                                    distinct++;
                                    px = B[0]; py = B[1]; pz = B[2];
                                }
                                cur = nx;
                            }
                            const double dx = fx - px, dy = fy - py, dz = fz - pz;
                            if (distinct > 1 && dx * dx + dy * dy + dz * dz <= eps2) distinct--;
                            else per += sqrt(dx * dx + dy * dy + dz * dz);
                            const double fa = 0.5 * sqrt(fax * fax + fay * fay + faz * faz);
                            order = distinct;
                            keep = distinct >= 3 && fa > eps * per;
                            vol += fv;
                            cx += (T)fcx; cy += (T)fcy; cz += (T)fcz;
                            farea = (T)fa;
                        }
                        if (!closed || steps < 3) bad = true;
                        if (keep) {
                            area += farea;
                            order_sum += order;
                            faces_kept++;
                            const int nid = nid_pre;
                            const int img = S.pimg[a];
                            const unsigned ib = ((unsigned)(imgc(img, 0) + 128) << 16) |
                                                ((unsigned)(imgc(img, 1) + 128) << 8) | (unsigned)(imgc(img, 2) + 128);
                            // canonical order: ascending neighbour id (walls first), then
                            // image; the face order rides in the low byte
                            const unsigned long long k = ((unsigned long long)((long long)nid + 8) << 32) |
                                                         ((unsigned long long)ib << 8) | (unsigned)(order & 0xff);
#pragma unroll
                            for (int r = 0; r < R; r++)
                                if (r == rnd) key[r] = k;
                        } else if (order >= 3) {
                            // a face dropped for its width (a sliver of distinct
                            // vertices) keeps its edges: they stay edges of the
                            // cell, held by the neighbouring faces
                            order_sum += order;
                        }
                    }
                    __syncwarp(gmask);
                }
                vol = gsum<G>(gmask, vol);
                cx = gsum<G>(gmask, cx); cy = gsum<G>(gmask, cy); cz = gsum<G>(gmask, cz);
                area = gsum<G>(gmask, area);
                const int nfk = __reduce_add_sync(gmask, faces_kept);
                const int osum = __reduce_add_sync(gmask, order_sum);
                bool anybad = __any_sync(gmask, bad);
                if (F32 && pass == 0 && !degen && !anybad) {
                    // FP32 vertex error ~ 3e-7 max(R, h) (h: the block side that
                    // bounds the stored FP32 offsets) relative to the thickness 3V/A
                    const float thick = (float)vol * rcp_a(2.f * (float)area);
                    const float scale = fmaxf(sqrt_a((float)r2), fmaxf(g.hf[0], fmaxf(g.hf[1], g.hf[2])));
                    if (!(thick * 10.f > scale)) {
                        if constexpr (HOT) {
                            // thin: FP64 statistics in the general kernel
                            if (gl == 0) {
                                const int slot = atomicAdd(o.retry0_count, 1);
                                o.retry0[slot] = i;
                            }
                            __syncwarp(gmask);
                            break;
                        }
                        degen = true;
                        __syncwarp(gmask);
                        continue;
                    }
                }
                int nv;
                // Weinberg codes: per slot s, byte s holds 1 + the slot of the
                // first earlier vertex this one coincides with (0: none)
                unsigned merged_into = 0;
                if (!HOT && degen) {
                    // distinct vertices: a vertex counts if no earlier one coincides
                    const double eps = pp.merge_rel * g.s, eps2 = eps * eps;
                    int cntv = 0;
#pragma unroll 1
                    for (int s = 0; s < VPL; s++) {
                        const int t = s * G + gl;
                        if (S.x.v.stri[t] != TRI_EMPTY) {
                            bool first = true;
                            int q = 0;
                            for (; q < t && first; q++) {
                                if (S.x.v.stri[q] == TRI_EMPTY) continue;
                                const double dx = S.x.v.dpos[q][0] - S.x.v.dpos[t][0], dy = S.x.v.dpos[q][1] - S.x.v.dpos[t][1],
                                             dz = S.x.v.dpos[q][2] - S.x.v.dpos[t][2];
                                if (dx * dx + dy * dy + dz * dz <= eps2) first = false;
                            }
                            if constexpr (TOPO) {
                                static_assert(VPL <= 4, "one byte a slot");
                                if (!first) merged_into |= (unsigned)q << (8 * s);  // q = match + 1
                            }
                            cntv += first;
                        }
                    }
                    nv = __reduce_add_sync(gmask, cntv);
                } else {
                    nv = T_;
                    if (nfk != T_ / 2 + 2) anybad = true;  // Euler with degree-3 vertices
                }
                if (anybad) {
                    fail = true;  // inconsistent topology: the FP64 big-cell tier redoes it
                } else {
                    // the cell's place in the face list, asked for before the sort
                    // so that the atomic's round trip overlaps it
                    long long fbase = 0;
                    if (gl == 0) fbase = (long long)atomicAdd(o.fcount, (unsigned long long)nfk);
                    // one round of faces: one key per lane, a shorter network
                    const bool one = HOT || F <= G;  // the hot kernel defers F > G
                    if (one) {
                        key[0] = bitonic1<G>(key[0], gl, gmask);
                    } else if constexpr (R == 2) {
                        bitonic2<G>(key[0], key[1], gl, gmask);
                    } else {
                        bitonic<R, G>(key, gl, gmask);
                    }
                    const int kstride = one ? 1 : R;
                    fbase = __shfl_sync(gmask, fbase, 0, G);
                    const bool overflow = fbase + nfk > o.fcap;
                    if (!overflow) {
#pragma unroll
                        for (int r = 0; r < R; r++) {
                            const int gpos = gl * kstride + r;
                            if (r < kstride && gpos < nfk) {
                                const unsigned long long k = key[r];
                                int2 ent;
                                ent.x = (int)((long long)(k >> 32) - 8);
                                const unsigned ib = (unsigned)(k >> 8) & 0xffffff;
                                ent.y = pack_img((int)((ib >> 16) & 0xff) - 128, (int)((ib >> 8) & 0xff) - 128,
                                                 (int)(ib & 0xff) - 128) |
                                        ((int)(k & 0xff) << 24);
                                o.faces[fbase + gpos] = ent;
                            }
                        }
                    }
                    if constexpr (TOPO) {
                        // the triangles by slot, for the Weinberg codes (tier 0: 64
                        // slots); the top byte names the vertex it merges into
#pragma unroll
                        for (int s = 0; s < VPL; s++) {
                            unsigned t = tri[s];
                            if (t != TRI_EMPTY) t = (t & 0xffffffu) | (((merged_into >> (8 * s)) & 0xffu) << 24);
                            o.topo[(long long)out_i * (G * VPL) + s * G + gl] = t;
                        }
                    }
                    if (gl == 0) {
                        const double v6 = vol;
                        o.vol[out_i] = v6 * (1.0 / 6.0);
                        if constexpr (F32) o.rfin[out_i] = sqrt_a(r2);
                        else o.rfin[out_i] = (float)sqrt(r2);
                        o.area[out_i] = (double)area;
                        // centroid = sum det (u0 + a + b) / (4 sum det)
                        const T inv = v6 != 0.0 ? (T)1 / ((T)4 * (T)v6) : (T)0;
                        o.cen[(long long)out_i * 3 + 0] = dref[0] + (double)(cx * inv);
                        o.cen[(long long)out_i * 3 + 1] = dref[1] + (double)(cy * inv);
                        o.cen[(long long)out_i * 3 + 2] = dref[2] + (double)(cz * inv);
                        o.nv[out_i] = nv;
                        o.ne[out_i] = osum / 2;
                        o.nf[out_i] = nfk;
                        o.status[out_i] = overflow ? (unsigned char)VG_CELL_CAP : (unsigned char)VG_CELL_OK;
                        if constexpr (TOPO) o.topo_n[out_i] = overflow ? 0 : T_;
                        o.fptr[out_i] = fbase;
                    }
                }
                __syncwarp(gmask);
                break;
                }  // pass
            } else if (!fail && gl == 0) {
                o.vol[out_i] = 0;
                o.area[out_i] = 0;
                o.rfin[out_i] = 0.f;
                for (int a = 0; a < 3; a++) o.cen[(long long)out_i * 3 + a] = 0;
                o.nv[out_i] = 0; o.ne[out_i] = 0; o.nf[out_i] = 0;
                o.status[out_i] = (unsigned char)status;
                o.fptr[out_i] = 0;
            }
            if (fail && gl == 0) {
                if (tier == 0 || tier == 3) {
                    const int slot = atomicAdd(o.retry_count, 1);
                    o.retry[slot] = i;
                } else if (tier == 1) {
                    const int slot = atomicAdd(o.retry2_count, 1);
                    o.retry2[slot] = i;
                }
                o.status[out_i] = VG_CELL_CAP;
                o.nf[out_i] = 0; o.nv[out_i] = 0; o.ne[out_i] = 0;
                o.vol[out_i] = 0; o.area[out_i] = 0; o.rfin[out_i] = 0.f;
                o.fptr[out_i] = 0;
            }
            if (pp.collect && gl == 0) {
                o.w_tested[out_i] = S.cnt[0];
                o.w_vtests[out_i] = S.cnt[1];
                o.w_cuts[out_i] = S.cnt[2];
                o.w_newv[out_i] = S.cnt[3];
                o.w_retest[out_i] = S.cnt[4];
                o.w_fallback[out_i] = (unsigned char)src.fell_back;
                o.w_pref[out_i] = S.cnt[5];
            }
            __syncwarp(gmask);
        }
    }
}

template <typename T, int VPL, int MAXP, bool BATCH, int G, bool TOPO = false, bool HOT = false>
cudaError_t launch_t(const Store &s, const Out &o, const Params &p, const Offsets &off, unsigned *ticket,
                     int sm_count, int warps, const int *cells, int ncells, int tier, cudaStream_t st) {
    const size_t smem = sizeof(Smem<T, VPL, MAXP, G, HOT>) * warps * (32 / G);
    auto kfn = k_cells3<T, VPL, MAXP, BATCH, G, TOPO, HOT>;
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // shared memory before L1: the resident CTAs are bounded by it
    e = cudaFuncSetAttribute(kfn, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, warps * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int grid = sm_count * per_sm;
    if (tier == 2) grid = sm_count;
    if ((e = cudaMemsetAsync(ticket, 0, sizeof(unsigned), st)) != cudaSuccess) return e;
    ++g_launch_count;
    kfn<<<grid, warps * 32, smem, st>>>(s, o, p, off, ticket, cells, ncells, tier);
    return cudaGetLastError();
}

}  // namespace

cudaError_t prefetch_rho(const Sys *sys, int nsys, const int *bstart, long long nblk, const float *kblock,
                         float kfixed, float *rho, cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    ++g_launch_count;
    k_prefetch_rho<<<(unsigned)((nblk + 255) / 256), 256, 0, st>>>(sys, nsys, bstart, nblk, kblock, kfixed, rho);
    return cudaGetLastError();
}

// Every tier runs one cell per warp (32 lanes); tier 0 holds cells up to 64
// vertices and 64 planes, tier 1 up to 128, tier 2 up to 256.
cudaError_t launch_cells3(const Store &s, const Out &o, const Params &p, const Offsets &off, int precision,
                          unsigned *ticket, int sm_count, int warps_per_cta, const int *cells, int ncells, int tier,
                          cudaStream_t st) {
    const int w = warps_per_cta > 0 ? min(warps_per_cta, VG_MAXT / 32) : VG_MAXT / 32;
    // the rare large cells (tiers 1, 2) always take the batched form
    if (tier == 2)
        return launch_t<double, 16, 256, true, 32>(s, o, p, off, ticket, sm_count, 1, cells, ncells, tier, st);
    if (tier == 1)
        return precision == VG_FP64
                   ? launch_t<double, 4, 128, true, 32>(s, o, p, off, ticket, sm_count, 2, cells, ncells, tier, st)
                   : launch_t<float, 4, 128, true, 32>(s, o, p, off, ticket, sm_count, 2, cells, ncells, tier, st);
    const bool batch = s.nsys > 1;
    if (precision == VG_FP64) {
        if (o.topo)  // the cells' triangles are kept for Weinberg codes (tier 0)
            return batch ? launch_t<double, VG_T0_VPL, 64, true, VG_T0_G, true>(s, o, p, off, ticket, sm_count, w, cells, ncells, tier, st)
                         : launch_t<double, VG_T0_VPL, 64, false, VG_T0_G, true>(s, o, p, off, ticket, sm_count, w, cells, ncells, tier, st);
        return batch ? launch_t<double, VG_T0_VPL, 64, true, VG_T0_G>(s, o, p, off, ticket, sm_count, w, cells, ncells, 0, st)
                     : launch_t<double, VG_T0_VPL, 64, false, VG_T0_G>(s, o, p, off, ticket, sm_count, w, cells, ncells, 0, st);
    }
    if (o.topo)  // the cells' triangles are kept for Weinberg codes (tier 0, or 3)
        return batch ? launch_t<float, VG_T0_VPL, 64, true, VG_T0_G, true>(s, o, p, off, ticket, sm_count, w, cells, ncells, tier, st)
                     : launch_t<float, VG_T0_VPL, 64, false, VG_T0_G, true>(s, o, p, off, ticket, sm_count, w, cells, ncells, tier, st);
    return batch ? launch_t<float, VG_T0_VPL, 64, true, VG_T0_G>(s, o, p, off, ticket, sm_count, w, cells, ncells, tier, st)
                 : launch_t<float, VG_T0_VPL, 64, false, VG_T0_G>(s, o, p, off, ticket, sm_count, w, cells, ncells, tier, st);
}

// The hot FP32 prefetch kernel over all cells (or a subset); the cells it
// defers go to o.retry0 for launch_cells3(..., tier 3).
cudaError_t launch_cells3_hot(const Store &s, const Out &o, const Params &p, const Offsets &off, unsigned *ticket,
                              int sm_count, int warps_per_cta, const int *cells, int ncells, cudaStream_t st) {
    const int w = warps_per_cta > 0 ? min(warps_per_cta, VG_MAXT / 32) : VG_MAXT / 32;
    if (o.topo)  // Weinberg codes: the triangles kept (one system only)
        return s.nsys > 1 ? cudaErrorInvalidValue
                          : launch_t<float, VG_T0_VPL, 64, false, VG_T0_G, true, true>(s, o, p, off, ticket, sm_count, w,
                                                                                       cells, ncells, 0, st);
    return s.nsys > 1
               ? launch_t<float, VG_T0_VPL, 64, true, VG_T0_G, false, true>(s, o, p, off, ticket, sm_count, w, cells,
                                                                           ncells, 0, st)
               : launch_t<float, VG_T0_VPL, 64, false, VG_T0_G, false, true>(s, o, p, off, ticket, sm_count, w, cells,
                                                                            ncells, 0, st);
}

}  // namespace vg
