// 2D cell kernel: a group of G lanes per Voronoi cell (polygon).
//
// The 2D method is the one of Sec. 2.1 (the paper explains it in 2D): the
// cell starts as the container rectangle relative to the particle
// (Eqs. 1-2) and is cut by the half-plane r.q > q.q/2 of each neighbour
// (Eq. 3; radical form with r_p^2 - r_q^2), visited near to far by the block
// walk of Sec. 2.1.3 and stopped by the radius bound.
//
// Representation: vertex (a, b) is where the boundary, running
// counter-clockwise, arrives along line a and leaves along line b.  A cut
// removes a contiguous run of vertices; for a removed vertex (x, y) the
// previous vertex is the one whose leaving line is x, so with the masks
// S = {leaving lines of removed vertices} and F = {arriving lines of removed
// vertices}, x not in S gives the new vertex (x, P) and y not in F gives the
// new vertex (P, y).  Exactly one of each exists; anything else is an
// inconsistency and the cell goes to the FP64 tier.  Statistics come from a
// shoelace sum over edges (vertex -> the vertex whose arriving line is its
// leaving line), one lane per vertex.
//
// FP32 form: coordinates relative to the particle in FP32; a vertex within
// the band tol32 * R * |q| (widened by its condition number) is re-solved
// from its two lines in FP64 and classified there.
#include "vg_internal.cuh"

namespace vg {
namespace {

constexpr unsigned EMPTY2 = 0xffffffffu;
constexpr int MAXP2 = 64;
constexpr float KAP0_2 = 4.0f;

template <typename T> struct P2;
template <> struct P2<float> { using t = float4; };
template <> struct P2<double> { using t = D4; };

__device__ __forceinline__ int imgc2(int img, int a) { return (int)(signed char)((img >> (8 * a)) & 0xff); }
__device__ __forceinline__ int pack2(int mx, int my) { return (mx & 0xff) | ((my & 0xff) << 8); }
__device__ __forceinline__ int la(unsigned v) { return v & 0xff; }
__device__ __forceinline__ int lb(unsigned v) { return (v >> 8) & 0xff; }
__device__ __forceinline__ unsigned mkv(int a, int b) { return (unsigned)a | ((unsigned)b << 8); }

struct CellC2 {
    int i, self_id, b[2];
    double p[2], rp;
    double rmax;  // largest radius of the cell's system (radical) or 0
    double hc;    // clipped cells: half the square side, 0 = none
};

template <typename T, int CAP>
struct Smem2 {
    typename P2<T>::t pl[MAXP2];  // line normal (x, y), constant (z)
    int pref[MAXP2], pimg[MAXP2];
    unsigned sv[CAP];
    T sx[CAP], sy[CAP];
    float sk[CAP];
    float4 mv[CAP];  // FP32 form: the cell's vertices (x, y, kappa, 0) by slot, free slots 0
    double dpos[CAP][2];
    unsigned char nxt[MAXP2];  // vertex slot by arriving line
    CellC2 cc;
    int cnt[4];
    Sys sysc;    // descriptor of the system of the current cell
    int sys_id;
};

// Block bound (Sec. 2.1.3) in 2D: a particle q cuts the cell only if some
// vertex v lies beyond its line, |q - v|^2 < |v|^2 (radical: + rmax^2 -
// r_p^2), so a block whose box [lo, hi] (relative to the particle) meets none
// of those discs holds no cutting particle.  Each disc is widened by sl * kappa
// (FP32 vertex error) and 1e-4 relative.  A free slot is (0, 0, 0): a disc of
// radius 0 (radical: sqrt(extra), which can only keep a block).
__device__ __noinline__ bool block_touches2(const float4 *mv, int n, float lo0, float lo1, float hi0, float hi1,
                                            float extra, float sl) {
    bool m = false;
#pragma unroll 1
    for (int t0 = 0; t0 < n; t0 += 8) {
#pragma unroll
        for (int t = t0; t < t0 + 8; t++) {
            const float4 v = mv[t];
            const float dx = fmaxf(0.f, fmaxf(lo0 - v.x, v.x - hi0));
            const float dy = fmaxf(0.f, fmaxf(lo1 - v.y, v.y - hi1));
            const float d2 = fmaf(dx, dx, dy * dy);
            const float rv = sqrt_a(fmaf(v.x, v.x, fmaf(v.y, v.y, extra))) + sl * v.z;
            m |= d2 < rv * rv * 1.0001f;
        }
    }
    return m;
}

template <int G>
__device__ __forceinline__ unsigned gballot(unsigned gmask, int gbase, bool p) {
    return (__ballot_sync(gmask, p) >> gbase) & (G == 32 ? 0xffffffffu : ((1u << G) - 1));
}
template <int G>
__device__ __forceinline__ int gscan(unsigned gmask, int gl, int v, int &total) {
    int x = v;
#pragma unroll
    for (int d = 1; d < G; d <<= 1) {
        int y = __shfl_up_sync(gmask, x, d, G);
        if (gl >= d) x += y;
    }
    total = __shfl_sync(gmask, x, G - 1, G);
    return x - v;
}
template <int G, typename V>
__device__ __forceinline__ V gsum(unsigned gmask, V v) {
#pragma unroll
    for (int d = G / 2; d > 0; d >>= 1) v += __shfl_xor_sync(gmask, v, d, G);
    return v;
}
template <int G, typename V>
__device__ __forceinline__ V gmax(unsigned gmask, V v) {
#pragma unroll
    for (int d = G / 2; d > 0; d >>= 1) {
        V o = __shfl_xor_sync(gmask, v, d, G);
        v = (o > v || o != o) ? o : v;  // a NaN wins on every lane alike
    }
    return v;
}
template <int G>
__device__ __forceinline__ unsigned long long gor64(unsigned gmask, unsigned long long v) {
    return ((unsigned long long)__reduce_or_sync(gmask, (unsigned)(v >> 32)) << 32) |
           __reduce_or_sync(gmask, (unsigned)v);
}

// Bitonic sort of G*E keys, E per lane (element gi = gl*E + e), inside a group.
template <int E, int G>
__device__ __forceinline__ void gbitonic(unsigned long long (&k)[E], int gl, unsigned gmask) {
#pragma unroll
    for (int size = 2; size <= G * E; size <<= 1) {
#pragma unroll
        for (int j = size >> 1; j > 0; j >>= 1) {
            if (j < E) {
#pragma unroll
                for (int e = 0; e < E; e++) {
                    if ((e & j) == 0) {
                        const int gi = gl * E + e;
                        const bool up = (gi & size) == 0;
                        const unsigned long long a = k[e], b = k[e ^ j];
                        if (up ? (a > b) : (a < b)) { k[e] = b; k[e ^ j] = a; }
                    }
                }
            } else {
                const int lm = j / E;
#pragma unroll
                for (int e = 0; e < E; e++) {
                    const int gi = gl * E + e;
                    const bool up = (gi & size) == 0;
                    const unsigned long long ot = __shfl_xor_sync(gmask, k[e], lm, G);
                    const bool keep_min = ((gi & j) == 0) == up;
                    const unsigned long long mn = k[e] < ot ? k[e] : ot, mx = k[e] < ot ? ot : k[e];
                    k[e] = keep_min ? mn : mx;
                }
            }
        }
    }
}

// FP64 line of a neighbour or of a wall (ref = -(1 + 2 axis + side)).
__device__ __forceinline__ void line64(const Grid &g, const Store &s, const CellC2 &c, int ref, int img, double n[2],
                                       double &cst) {
    if (ref < 0) {
        const int w = -ref - 1, a = w >> 1, side = w & 1;
        n[0] = n[1] = 0.0;
        n[a] = side ? 1.0 : -1.0;
        cst = side ? __dsub_rn(g.hi[a], c.p[a]) : __dsub_rn(c.p[a], g.lo[a]);
        // a clipped cell's square side (on a periodic axis every wall is one)
        if (c.hc > 0.0 && (g.per[a] || c.hc < cst)) cst = c.hc;
        return;
    }
    const D4 q = s.p64[ref];
    const double qa[2] = {q.x, q.y};
    double qq = 0.0;
#pragma unroll
    for (int a = 0; a < 2; a++) {
        n[a] = __dsub_rn(__dadd_rn(qa[a], __dmul_rn((double)imgc2(img, a), g.L[a])), c.p[a]);
        qq = __dadd_rn(qq, __dmul_rn(n[a], n[a]));
    }
    cst = __dmul_rn(0.5, __dsub_rn(__dadd_rn(qq, __dmul_rn(c.rp, c.rp)), __dmul_rn(q.w, q.w)));
}

__device__ __noinline__ void vertex64_2(const Grid *g, const Store *st, const CellC2 *c, const int *pref,
                                        const int *pimg, unsigned v, double *out) {
    double n1[2], n2[2], c1, c2;
    line64(*g, *st, *c, pref[la(v)], pimg[la(v)], n1, c1);
    line64(*g, *st, *c, pref[lb(v)], pimg[lb(v)], n2, c2);
    const double det = n1[0] * n2[1] - n1[1] * n2[0];
    out[0] = (c1 * n2[1] - c2 * n1[1]) / det;
    out[1] = (n1[0] * c2 - n2[0] * c1) / det;
}

__device__ __noinline__ int classify64_2(const Grid *g, const Store *st, const CellC2 *c, const int *pref,
                                         const int *pimg, unsigned v, int ref, int img, double tau_rel_s) {
    double p[2], n[2], cst;
    vertex64_2(g, st, c, pref, pimg, v, p);
    line64(*g, *st, *c, ref, img, n, cst);
    const double tau = tau_rel_s * sqrt(n[0] * n[0] + n[1] * n[1]);
    const double d = __dsub_rn(__dadd_rn(__dmul_rn(n[0], p[0]), __dmul_rn(n[1], p[1])), cst);
    return d > tau ? 1 : (d >= -tau ? 0 : -1);
}

// FP32 intersection of two lines; condition number returned in kap.
template <typename T>
__device__ __forceinline__ void meet(typename P2<T>::t A, T bx, T by, T bc, T &x, T &y, float &kap) {
    const T det = A.x * by - A.y * bx;
    const float m = (float)((A.x * A.x + A.y * A.y) * (bx * bx + by * by));
    if constexpr (sizeof(T) == 4) {
        const float id = rcp_a(det);
        x = (A.z * by - bc * A.y) * id;
        y = (A.x * bc - bx * A.z) * id;
        kap = fmaxf(1.f, sqrt_a(m) * fabsf(id) * (1.f / KAP0_2));
    } else {
        x = (A.z * by - bc * A.y) / det;
        y = (A.x * bc - bx * A.z) / det;
        kap = fmaxf(1.f, sqrtf(m) / (fabsf((float)det) * KAP0_2));
    }
}

// resident 128-thread CTAs per SM the register budget is sized for (four:
// 128 registers, where ptxas also spills least)
#ifndef VG2_MINB
#define VG2_MINB 4
#endif

template <typename T, int G, int CAP, bool BATCH>
__global__ void __launch_bounds__(128, VG2_MINB) k_cells2(const __grid_constant__ Store st,
                                                const __grid_constant__ Out o, const __grid_constant__ Params pp,
                                                const __grid_constant__ Offsets off, unsigned *ticket,
                                                const int *cells, int ncells, int tier) {
    constexpr bool F32 = sizeof(T) == 4;
    constexpr int VPL = CAP / G;
    constexpr int GPW = 32 / G;  // groups per warp
    using S_t = Smem2<T, CAP>;
    extern __shared__ __align__(32) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gid = lane / G, gl = lane % G, gbase = gid * G;
    const unsigned gmask = G == 32 ? FULL : (((1u << G) - 1) << gbase);
    S_t &S = reinterpret_cast<S_t *>(smem_raw)[warp * GPW + gid];
    const int total = cells ? (tier == 1 ? *o.retry_count : (tier == 2 ? *o.retry2_count : ncells)) : st.n;
    const float tol32f = (float)pp.tol32;
    if (gl == 0) S.sys_id = -1;
    __syncwarp(gmask);
    const Sys &SY = sys_ref<BATCH>(st, S.sysc);
    const Grid &g = SY.g;

    for (int iter = 0; iter < (1 << 30); iter++) {
        int i = 0;
        if (gl == 0) i = (int)atomicAdd(ticket, 1u);
        i = __shfl_sync(gmask, i, 0, G);
        if (i >= total) break;
        if (cells) i = cells[i];
        // ---------------------------------------------------------------- setup
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
        }
        const double tau_rel_s = pp.tau_rel * g.s;
        const int kh = __ldg(&st.sblk[i]) - (int)SY.blk_base;
        const float4 p32 = __ldg(&st.p32[i]);
        const float o0 = p32.x, o1 = p32.y;
        if (gl == 0) {
            const D4 p64 = st.p64[i];
            S.cc.i = i;
            S.cc.self_id = __ldg(&st.sid[i]);
            S.cc.b[0] = kh % g.nb[0];
            S.cc.b[1] = kh / g.nb[0];
            S.cc.p[0] = p64.x; S.cc.p[1] = p64.y;
            S.cc.rp = p64.w;
            S.cc.rmax = st.radical ? (BATCH ? S.sysc.rmax : st.sys[0].rmax) : 0.0;
            S.cc.hc = 0.5 * pp.clip;
            S.cnt[0] = S.cnt[1] = S.cnt[2] = S.cnt[3] = 0;
        }
        __syncwarp(gmask);
        const int b0 = S.cc.b[0], b1 = S.cc.b[1];
        // --------------------------------------------- initial rectangle, Eqs. 1-2
        unsigned v[VPL];
        T vx[VPL], vy[VPL];
        float kap[VPL];
        {
            T lo[2], hi[2];
            const float oo[2] = {o0, o1};
            const int bb[2] = {b0, b1};
#pragma unroll
            for (int a = 0; a < 2; a++) {
                if (g.per[a]) {
                    lo[a] = (T)(-0.5) * (T)(F32 ? (double)g.Lf[a] : g.L[a]);
                    hi[a] = -lo[a];
                } else if constexpr (F32) {
                    lo[a] = -((float)bb[a] * g.hf[a] + oo[a]);
                    hi[a] = (float)(g.nb[a] - bb[a]) * g.hf[a] - oo[a];
                } else {
                    lo[a] = g.lo[a] - S.cc.p[a];
                    hi[a] = g.hi[a] - S.cc.p[a];
                }
            }
            // clipped cells (Sec. 3.1.3): the box meets the square of side clip
            // around the particle; on a periodic axis a square smaller than the
            // period replaces the self-image lines by walls
            if (pp.clip > 0.0) {
                const T hc = (T)(0.5 * pp.clip);
#pragma unroll
                for (int a = 0; a < 2; a++) {
                    if (g.per[a]) {
                        if (pp.clip < g.L[a]) { lo[a] = -hc; hi[a] = hc; }
                    } else {
                        lo[a] = lo[a] > -hc ? lo[a] : -hc;
                        hi[a] = hi[a] < hc ? hi[a] : hc;
                    }
                }
            }
            if (gl < 4) {
                // lines: 0 x-, 1 x+, 2 y-, 3 y+
                const int a = gl >> 1, side = gl & 1;
                T n[2] = {0, 0};
                T c;
                int ref, img;
                if (g.per[a] && !(pp.clip > 0.0 && pp.clip < g.L[a])) {
                    const T L = F32 ? (T)g.Lf[a] : (T)g.L[a];
                    n[a] = side ? L : -L;
                    c = (T)0.5 * L * L;
                    ref = i;
                    img = pack2(a == 0 ? (side ? 1 : -1) : 0, a == 1 ? (side ? 1 : -1) : 0);
                } else {
                    n[a] = side ? (T)1 : (T)-1;
                    c = side ? hi[a] : -lo[a];
                    ref = -(1 + 2 * a + side);
                    img = 0;
                }
                typename P2<T>::t P;
                P.x = n[0]; P.y = n[1]; P.z = c; P.w = 0;
                S.pl[gl] = P;
                S.pref[gl] = ref;
                S.pimg[gl] = img;
            }
#pragma unroll
            for (int s = 0; s < VPL; s++) { v[s] = EMPTY2; vx[s] = vy[s] = (T)0; kap[s] = 1.f; }
            if (gl < 4) {
                // counter-clockwise: (x-,y-) (y-,x+) (x+,y+) (y+,x-)
                const unsigned tv[4] = {mkv(0, 2), mkv(2, 1), mkv(1, 3), mkv(3, 0)};
                const T px[4] = {lo[0], hi[0], hi[0], lo[0]}, py[4] = {lo[1], lo[1], hi[1], hi[1]};
                v[0] = tv[gl];
                vx[0] = px[gl];
                vy[0] = py[gl];
            }
            if constexpr (F32) {
#pragma unroll
                for (int s = 0; s < VPL; s++)
                    S.mv[s * G + gl] = v[s] != EMPTY2 ? make_float4(vx[s], vy[s], kap[s], 0.f)
                                                       : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        int nvert = 4;
        unsigned rows = 1;
        unsigned long long live = 0xfull;
        T r2 = gmax<G>(gmask, gl < 4 ? vx[0] * vx[0] + vy[0] * vy[0] : (T)0);
        int flags = 0;  // 1 degenerate, 2 failure, 4 empty, 8 duplicate
        int limit = 0;
        float eqm = 0.f;  // FP32: largest position error of the candidates so far
        // FP32: that error moves |q| and R by about eqm and the vertices by
        // kappa eqm; 64 eqm R covers a small cell
        auto stop2 = [&]() -> T {
            const T margin = F32 ? (T)1.0001 : (T)(1.0 + 1e-12);
            const T ea = F32 ? (T)(64.f * eqm) : (T)0;
            if (!st.radical) return (T)4 * r2 * margin + ea * sqrt(r2);
            const T disc = r2 + (T)(S.cc.rmax * S.cc.rmax) - (T)(S.cc.rp * S.cc.rp);
            if (disc <= (T)0) return (T)0;
            const T rs = sqrt(r2) + sqrt(disc);
            return rs * rs * margin + ea * rs;
        };
        __syncwarp(gmask);
        T stop = stop2();

        // ------------------------------------------- walk (Sec. 2.1.3), per block
        const float hmin = fminf(g.hf[0], g.hf[1]), hmax = fmaxf(g.hf[0], g.hf[1]);
        // shell s has 8 s blocks: up to 16000 shells the walk (about 4 s^2
        // steps) ends before its guard of 2^30 steps
        const int maxs = min(16000, SY.off_shell + 4 + 2 * max(g.nb[0], g.nb[1]));
        const int ocount = SY.off_count, obase = SY.off_base;
        int e = 0, shell = 0, sidx = 0, mode = 1;  // 1 list, 2 shells, 3 done
        // blocks are taken G at a time, one per lane of the group (a window):
        // each lane resolves its block and loads its particle range, so the
        // loads of a window are in flight together; the blocks that hold
        // particles are then cut one after another
        for (int guard = 0; guard < (1 << 30) && mode != 3 && !(flags & 6); guard++) {
            int wox = 0, woy = 0;
            bool cand = false, last = false;
            if (mode == 1) {
                if (e >= ocount) { mode = 2; shell = 1; sidx = 0; continue; }
                const int ei = e + gl;
                bool beyond = true;
                if (ei < ocount) {
                    const float lbv = __ldg(&off.lb[obase + ei]);
                    beyond = (T)(lbv * lbv) * (T)0.99998 >= stop;
                    const int code = __ldg(&off.code[obase + ei]);
                    wox = imgc2(code, 0);
                    woy = imgc2(code, 1);
                }
                // the list is sorted by its bound: entries past the first one
                // beyond the stop radius are all beyond it
                const unsigned bb = gballot<G>(gmask, gbase, beyond);
                const int first = bb ? __ffs(bb) - 1 : G;
                cand = gl < first;
                last = first < G && e + first < ocount;
                e += G;
            } else {
                const float sb = (float)(shell - 1) * hmin;
                if ((T)(sb * sb) * (T)0.99998 >= stop) { mode = 3; continue; }
                if (shell > maxs) { limit = 1; mode = 3; continue; }
                // the shell's surface only: two rows of wd, two columns of wd - 2
                const int wd = 2 * shell + 1, ns = 4 * wd - 4;
                if (sidx >= ns) { shell++; sidx = 0; continue; }
                const int si = sidx + gl;
                if (si < ns) {
                    if (si < 2 * wd) {
                        const int r = si < wd ? si : si - wd;
                        wox = r - shell;
                        woy = si < wd ? -shell : shell;
                    } else {
                        const int t = si - 2 * wd, r = t < wd - 2 ? t : t - (wd - 2);
                        wox = t < wd - 2 ? -shell : shell;
                        woy = r - (shell - 1);
                    }
                    // shell members that the offset list did not hold (its bound is
                    // below off_shell * h_min, in FP32, exactly as the list was cut)
                    const float lbmax = (float)SY.off_shell * hmin;
                    const float lbx = fmaxf(0.f, (float)(abs(wox) - 1)) * g.hf[0];
                    const float lby = fmaxf(0.f, (float)(abs(woy) - 1)) * g.hf[1];
                    cand = !(lbx * lbx + lby * lby < lbmax * lbmax);
                }
                sidx += G;
            }
            // each lane's block: resolve, distance bound, particle range
            int wj0 = 0, wj1 = 0, wimg = 0;
            if (cand) {
                int t0 = b0 + wox, t1 = b1 + woy, m0 = 0, m1 = 0;
                if (g.per[0]) { m0 = floordiv_near(t0, g.nb[0]); t0 -= m0 * g.nb[0]; }
                else if (t0 < 0 || t0 >= g.nb[0]) cand = false;
                if (g.per[1]) { m1 = floordiv_near(t1, g.nb[1]); t1 -= m1 * g.nb[1]; }
                else if (t1 < 0 || t1 >= g.nb[1]) cand = false;
                if (cand) {
                    const float lo0 = (float)wox * g.hf[0] - o0, lo1 = (float)woy * g.hf[1] - o1;
                    const float gx = lo0 > 0.f ? lo0 : (lo0 + g.hf[0] < 0.f ? -(lo0 + g.hf[0]) : 0.f);
                    const float gy = lo1 > 0.f ? lo1 : (lo1 + g.hf[1] < 0.f ? -(lo1 + g.hf[1]) : 0.f);
                    cand = !((T)(gx * gx + gy * gy) * (T)0.99998 >= stop);
                }
                if (cand) {
                    const int kb = (int)SY.blk_base + t0 + g.nb[0] * t1;
                    wj0 = __ldg(&st.bstart[kb]);
                    wj1 = __ldg(&st.bstart[kb + 1]);
                    wimg = pack2(m0, m1);
                    cand = wj1 > wj0;
                    if constexpr (F32) {
                        // beyond the offset list (extended cells): the block bound,
                        // for blocks whose particles would cost more than the test
                        if (cand && mode == 2 && wj1 - wj0 >= 8) {
                            const float bl0 = (float)wox * g.hf[0] - o0, bl1 = (float)woy * g.hf[1] - o1;
                            const float ex = st.radical ? (float)(S.cc.rmax * S.cc.rmax - S.cc.rp * S.cc.rp) : 0.f;
                            const float sl = 1e-5f * (sqrt_a((float)r2) + hmax);
                            cand = block_touches2(S.mv, G * (32 - __clz(rows)), bl0, bl1, bl0 + g.hf[0],
                                                  bl1 + g.hf[1], fmaxf(ex, 0.f), sl);
                        }
                    }
                }
            }
            if (last) mode = 3;  // after this window
            unsigned blocks = gballot<G>(gmask, gbase, cand);
            while (blocks && !(flags & 6)) {
                const int bl = __ffs(blocks) - 1;
                blocks &= blocks - 1;
                const int ox = __shfl_sync(gmask, wox, bl, G), oy = __shfl_sync(gmask, woy, bl, G);
                const int j0 = __shfl_sync(gmask, wj0, bl, G), j1 = __shfl_sync(gmask, wj1, bl, G);
                const int img = __shfl_sync(gmask, wimg, bl, G);
                const int m0 = imgc2(img, 0), m1 = imgc2(img, 1);
                {
                    // cuts of earlier blocks may have brought the bound closer
                    const float lo0 = (float)ox * g.hf[0] - o0, lo1 = (float)oy * g.hf[1] - o1;
                    const float gx = lo0 > 0.f ? lo0 : (lo0 + g.hf[0] < 0.f ? -(lo0 + g.hf[0]) : 0.f);
                    const float gy = lo1 > 0.f ? lo1 : (lo1 + g.hf[1] < 0.f ? -(lo1 + g.hf[1]) : 0.f);
                    if ((T)(gx * gx + gy * gy) * (T)0.99998 >= stop) continue;
                }
            for (int jb = j0; jb < j1 && !(flags & 6); jb += G) {
                const int j = jb + gl;
                T qx = 0, qy = 0, qq = 0, rj = 0;
                bool ok = false;
                if (j < j1) {
                    if constexpr (F32) {
                        const float4 pj = __ldg(&st.p32[j]);
                        qx = __fadd_rn(__fmul_rn((float)ox, g.hf[0]), __fsub_rn(pj.x, o0));
                        qy = __fadd_rn(__fmul_rn((float)oy, g.hf[1]), __fsub_rn(pj.y, o1));
                        qq = __fadd_rn(__fmul_rn(qx, qx), __fmul_rn(qy, qy));
                        rj = pj.w;
                    } else {
                        const D4 pj = st.p64[j];
                        qx = __dsub_rn(__dadd_rn(pj.x, __dmul_rn((double)m0, g.L[0])), S.cc.p[0]);
                        qy = __dsub_rn(__dadd_rn(pj.y, __dmul_rn((double)m1, g.L[1])), S.cc.p[1]);
                        qq = __dadd_rn(__dmul_rn(qx, qx), __dmul_rn(qy, qy));
                        rj = pj.w;
                    }
                    ok = !(ox == 0 && oy == 0 && j == i) && qq < stop;
                }
                unsigned want = gballot<G>(gmask, gbase, ok);
                while (want) {
                    const int src = __ffs(want) - 1;
                    want &= want - 1;
                    const T cx = __shfl_sync(gmask, qx, src, G), cy = __shfl_sync(gmask, qy, src, G);
                    const T cq = __shfl_sync(gmask, qq, src, G), cr = __shfl_sync(gmask, rj, src, G);
                    const int ref = jb + src;
                    if (cq >= stop) continue;
                    // coincident: in FP32 perhaps only after rounding, so a retry
                    if (cq < (T)1e-30) { flags |= F32 ? 2 : 8; continue; }
                    const T c = st.radical ? (T)0.5 * (cq + (T)(S.cc.rp * S.cc.rp) - cr * cr) : (T)0.5 * cq;
                    // ---------------------------------------- cut by q.r = c
                    if (pp.collect && gl == 0) { S.cnt[0]++; S.cnt[1] += nvert; }
                    T tau;
                    if constexpr (F32) {
                        // block-relative FP32 positions are off by a few units in
                        // the last place of the block side, more with the block
                        // offset; tiny cells need that absolute error in the band
                        eqm = fmaxf(eqm, 1.2e-7f * (float)(abs(ox) + abs(oy) + 2) * hmax);
                        const float rq = sqrt_a(cq);
                        tau = tol32f * sqrt_a(r2) * rq + eqm * (sqrt_a(r2) + 2.f * rq);
                    }
                    else tau = (T)(tau_rel_s * sqrt((double)cq));
                    unsigned outm = 0, nearm = 0, onm = 0;
#pragma unroll
                    for (int s = 0; s < VPL; s++) {
                        if (((rows >> s) & 1) && v[s] != EMPTY2) {
                            const T d = vx[s] * cx + vy[s] * cy - c;
                            const T band = F32 ? tau * (T)kap[s] : tau;
                            if (d > band) outm |= 1u << s;
                            else if (d >= -band) {
                                if (F32) nearm |= 1u << s;
                                else onm |= 1u << s;
                            }
                        }
                    }
                    if constexpr (F32) {
                        if (__any_sync(gmask, nearm)) {
                            if (pp.collect && gl == 0) S.cnt[3]++;
#pragma unroll
                            for (int s = 0; s < VPL; s++) {
                                if (nearm & (1u << s)) {
                                    const int r = classify64_2(&g, &st, &S.cc, S.pref, S.pimg, v[s], ref, img, tau_rel_s);
                                    if (r > 0) outm |= 1u << s;
                                    else if (r == 0) onm |= 1u << s;
                                }
                            }
                        }
                    }
                    if (!__any_sync(gmask, outm)) continue;
                    if (__any_sync(gmask, onm)) flags |= 1;
                    if (pp.collect && gl == 0) S.cnt[2]++;
                    // removed vertices: masks of their arriving and leaving lines
                    unsigned long long Fm = 0, Sm = 0;
                    int kept = 0;
#pragma unroll
                    for (int s = 0; s < VPL; s++) {
                        if (outm & (1u << s)) {
                            Fm |= 1ull << la(v[s]);
                            Sm |= 1ull << lb(v[s]);
                        } else if (v[s] != EMPTY2) {
                            kept++;
                        }
                    }
                    Fm = gor64<G>(gmask, Fm);
                    Sm = gor64<G>(gmask, Sm);
                    kept = __reduce_add_sync(gmask, kept);
                    // no vertex left: an empty power cell, but for a Voronoi cell
                    // (which holds its particle) a numerical failure
                    if (kept == 0) { flags |= st.radical ? 4 : 2; break; }
                    const unsigned long long freep = ~live;
                    if (!freep) { flags |= 2; break; }
                    const int np = __ffsll((long long)freep) - 1;
                    if (np >= MAXP2) { flags |= 2; break; }
                    // the lanes holding the run's ends make the two new vertices;
                    // each lies on an old edge, so within the old radius (a vertex
                    // beyond it, or not finite, is a numerical failure)
                    int nA = 0, nB = 0;
                    bool wild = false;
                    const T r2lim = r2 * (T)1.01;
#pragma unroll
                    for (int s = 0; s < VPL; s++) {
                        if (outm & (1u << s)) {
                            const int x = la(v[s]), y = lb(v[s]);
                            if (!((Sm >> x) & 1)) {
                                // (x, P): on line x and the cutting line
                                T nx, ny;
                                float kp;
                                meet<T>(S.pl[x], cx, cy, c, nx, ny, kp);
                                S.sv[0] = mkv(x, np); S.sx[0] = nx; S.sy[0] = ny; S.sk[0] = kp;
                                wild |= !(nx * nx + ny * ny <= r2lim);
                                nA++;
                            }
                            if (!((Fm >> y) & 1)) {
                                T nx, ny;
                                float kp;
                                meet<T>(S.pl[y], cx, cy, c, nx, ny, kp);
                                S.sv[1] = mkv(np, y); S.sx[1] = nx; S.sy[1] = ny; S.sk[1] = kp;
                                wild |= !(nx * nx + ny * ny <= r2lim);
                                nB++;
                            }
                            v[s] = EMPTY2;
                        }
                    }
                    nA = __reduce_add_sync(gmask, nA);
                    nB = __reduce_add_sync(gmask, nB);
                    wild = __any_sync(gmask, wild);
                    if (nA != 1 || nB != 1 || wild || kept + 2 > CAP) { flags |= 2; break; }
                    if (gl == 0) {
                        typename P2<T>::t P;
                        P.x = cx; P.y = cy; P.z = c; P.w = 0;
                        S.pl[np] = P;
                        S.pref[np] = ref;
                        S.pimg[np] = img;
                    }
                    __syncwarp(gmask);
                    // free slots take the two new vertices in order
                    int rank0 = 0;
                    unsigned long long lv = 0;
                    T rr = 0;
                    rows = 0;
#pragma unroll
                    for (int s = 0; s < VPL; s++) {
                        const bool fr = v[s] == EMPTY2;
                        const unsigned fm = gballot<G>(gmask, gbase, fr);
                        const int rank = rank0 + __popc(fm & ((1u << gl) - 1));
                        rank0 += __popc(fm);
                        if (fr && rank < 2) {
                            v[s] = S.sv[rank];
                            vx[s] = S.sx[rank]; vy[s] = S.sy[rank];
                            kap[s] = S.sk[rank];
                        }
                        if (v[s] != EMPTY2) {
                            lv |= (1ull << la(v[s])) | (1ull << lb(v[s]));
                            T q2 = vx[s] * vx[s] + vy[s] * vy[s];
                            if constexpr (F32) q2 *= 1.f + 4e-6f * kap[s];
                            rr = rr > q2 ? rr : q2;
                        }
                        if constexpr (F32)
                            S.mv[s * G + gl] = v[s] != EMPTY2 ? make_float4(vx[s], vy[s], kap[s], 0.f)
                                                               : make_float4(0.f, 0.f, 0.f, 0.f);
                        if (__any_sync(gmask, v[s] != EMPTY2)) rows |= 1u << s;
                    }
                    live = gor64<G>(gmask, lv);
                    r2 = gmax<G>(gmask, rr);
                    nvert = kept + 2;
                    __syncwarp(gmask);
                    stop = stop2();
                }
            }
            }  // blocks of the window
        }

        if (mode != 3 && !(flags & 6)) limit = 1;  // the guard ran out

        // ------------------------------------------------------------ statistics
        int status = VG_CELL_OK;
        bool fail = flags & 2;
        if (flags & 4) status = VG_CELL_EMPTY;
        else if (flags & 8) status = VG_CELL_DUP;
        else if (limit) status = VG_CELL_LIMIT;
        const int out_i = S.cc.self_id;
        bool degen = flags & 1;
        if constexpr (F32) {
            // an ill-conditioned vertex (kappa >= 64) is off by more than the
            // 1e-5 bar allows: the statistics take FP64 vertices
            bool hk = false;
#pragma unroll
            for (int s = 0; s < VPL; s++) hk |= v[s] != EMPTY2 && kap[s] >= 64.f;
            const bool anyhk = __any_sync(gmask, hk);
            degen = degen || anyhk;
        }
        if (!fail && status == VG_CELL_OK) {
            // reference point: a vertex of the cell (fans from a far particle
            // cancel); radical cells small against that distance use FP64
            T rx = 0, ry = 0;
            {
                int rsl = 0;
                unsigned occ = gballot<G>(gmask, gbase, v[0] != EMPTY2);
#pragma unroll
                for (int s = 1; s < VPL; s++) {
                    const unsigned oc = gballot<G>(gmask, gbase, v[s] != EMPTY2);
                    if (!occ && oc) { occ = oc; rsl = s; }
                }
                const int rl = __ffs(occ) - 1;
                T cand_x = 0, cand_y = 0;
#pragma unroll
                for (int s = 0; s < VPL; s++)
                    if (s == rsl) { cand_x = vx[s]; cand_y = vy[s]; }
                rx = __shfl_sync(gmask, cand_x, rl, G);
                ry = __shfl_sync(gmask, cand_y, rl, G);
            }
            // pass 0 sums the FP32 vertices; a cell thin against its distance
            // from the particle gets a pass from FP64 vertices
            for (int pass = 0; pass < 2; pass++) {
#pragma unroll
            for (int s = 0; s < VPL; s++) {
                const int t = s * G + gl;
                S.sv[t] = v[s];
                S.sx[t] = vx[s];
                S.sy[t] = vy[s];
                if (v[s] != EMPTY2) {
                    S.nxt[la(v[s])] = (unsigned char)t;
                    if (degen) {
                        if constexpr (F32) vertex64_2(&g, &st, &S.cc, S.pref, S.pimg, v[s], S.dpos[t]);
                        else { S.dpos[t][0] = vx[s]; S.dpos[t][1] = vy[s]; }
                    }
                }
            }
            __syncwarp(gmask);
            const double eps = pp.merge_rel * g.s, eps2 = eps * eps;
            double area = 0.0;
            T cxs = 0, cys = 0, per = 0;
            int edges = 0;
            bool bad = false;
            unsigned long long key[VPL];
#pragma unroll
            for (int s = 0; s < VPL; s++) {
                key[s] = ~0ull;
                if (v[s] == EMPTY2) continue;
                const int bl = lb(v[s]);
                const int nx = S.nxt[bl];
                if (nx >= CAP || S.sv[nx] == EMPTY2 || la(S.sv[nx]) != bl) { bad = true; continue; }
                bool keep = true;
                if (!degen) {
                    const T ax = vx[s] - rx, ay = vy[s] - ry, bx = S.sx[nx] - rx, by = S.sy[nx] - ry;
                    const T cr = ax * by - ay * bx;
                    area += (double)cr;
                    cxs += (ax + bx) * cr;
                    cys += (ay + by) * cr;
                    const T l2 = (bx - ax) * (bx - ax) + (by - ay) * (by - ay);
                    if constexpr (F32) per += sqrt_a(l2);
                    else per += sqrt(l2);
                } else {
                    const double ax = S.dpos[s * G + gl][0] - (double)rx, ay = S.dpos[s * G + gl][1] - (double)ry;
                    const double bx = S.dpos[nx][0] - (double)rx, by = S.dpos[nx][1] - (double)ry;
                    const double cr = ax * by - ay * bx;
                    area += cr;
                    cxs += (T)((ax + bx) * cr);
                    cys += (T)((ay + by) * cr);
                    const double l2 = (bx - ax) * (bx - ax) + (by - ay) * (by - ay);
                    per += (T)sqrt(l2);
                    keep = l2 > eps2;  // a zero-length edge is no neighbour
                }
                if (keep) {
                    edges++;
                    const int ref = S.pref[bl];
                    const int nid = ref >= 0 ? __ldg(&st.sid[ref]) : ref;
                    const int im = S.pimg[bl];
                    const unsigned ib = ((unsigned)(imgc2(im, 0) + 128) << 16) | ((unsigned)(imgc2(im, 1) + 128) << 8) | 128u;
                    key[s] = ((unsigned long long)((long long)nid + 8) << 32) | ((unsigned long long)ib << 8) | 2u;
                }
            }
            area = gsum<G>(gmask, area);
            cxs = gsum<G>(gmask, cxs);
            cys = gsum<G>(gmask, cys);
            per = gsum<G>(gmask, per);
            edges = __reduce_add_sync(gmask, edges);
            const bool anybad = __any_sync(gmask, bad) || !(area > 0.0);
            if (F32 && pass == 0 && !degen && !anybad) {
                // FP32 vertex error ~ 3e-7 max(R, h) (h: the block side that
                // bounds the stored FP32 offsets) relative to the thickness 2A/P
                const float thick = (float)area * rcp_a((float)per);
                const float scale = fmaxf(sqrt_a((float)r2), fmaxf(g.hf[0], g.hf[1]));
                if (!(thick * 10.f > scale)) {
                    degen = true;
                    __syncwarp(gmask);
                    continue;
                }
            }
            if (anybad) {
                fail = true;
            } else {
                // each lane's keys sorted across the group
                unsigned long long kk[VPL];
#pragma unroll
                for (int s = 0; s < VPL; s++) kk[s] = key[s];
                gbitonic<VPL, G>(kk, gl, gmask);
                long long fbase = 0;
                if (gl == 0) fbase = (long long)atomicAdd(o.fcount, (unsigned long long)edges);
                fbase = __shfl_sync(gmask, fbase, 0, G);
                const bool overflow = fbase + edges > o.fcap;
                if (!overflow) {
#pragma unroll
                    for (int s = 0; s < VPL; s++) {
                        const int gpos = gl * VPL + s;
                        if (gpos < edges) {
                            const unsigned long long k = kk[s];
                            int2 ent;
                            ent.x = (int)((long long)(k >> 32) - 8);
                            const unsigned ib = (unsigned)(k >> 8) & 0xffffff;
                            ent.y = pack2((int)((ib >> 16) & 0xff) - 128, (int)((ib >> 8) & 0xff) - 128) | (2 << 24);
                            o.faces[fbase + gpos] = ent;
                        }
                    }
                }
                if (gl == 0) {
                    o.vol[out_i] = 0.5 * area;
                    if constexpr (F32) o.rfin[out_i] = sqrtf(r2);
                    else o.rfin[out_i] = (float)sqrt(r2);
                    o.area[out_i] = (double)per;
                    const T inv = (T)1 / ((T)3 * (T)area);
                    o.cen[(long long)out_i * 3 + 0] = (double)rx + (double)(cxs * inv);
                    o.cen[(long long)out_i * 3 + 1] = (double)ry + (double)(cys * inv);
                    o.cen[(long long)out_i * 3 + 2] = 0.0;
                    o.nv[out_i] = edges;
                    o.ne[out_i] = edges;
                    o.nf[out_i] = edges;
                    o.status[out_i] = overflow ? (unsigned char)VG_CELL_CAP : (unsigned char)VG_CELL_OK;
                    o.fptr[out_i] = fbase;
                }
            }
            break;
            }  // pass
        } else if (!fail && gl == 0) {
            o.vol[out_i] = 0; o.area[out_i] = 0; o.rfin[out_i] = 0.f;
            for (int a = 0; a < 3; a++) o.cen[(long long)out_i * 3 + a] = 0;
            o.nv[out_i] = o.ne[out_i] = o.nf[out_i] = 0;
            o.status[out_i] = (unsigned char)status;
            o.fptr[out_i] = 0;
        }
        if (fail && gl == 0) {
            if (tier == 0) {
                const int slot = atomicAdd(o.retry_count, 1);
                o.retry[slot] = i;
            } else if (tier == 1) {
                const int slot = atomicAdd(o.retry2_count, 1);
                o.retry2[slot] = i;
            }
            o.status[out_i] = VG_CELL_CAP;
            o.nv[out_i] = o.ne[out_i] = o.nf[out_i] = 0;
            o.vol[out_i] = 0; o.area[out_i] = 0; o.rfin[out_i] = 0.f;
            o.fptr[out_i] = 0;
        }
        if (pp.collect && gl == 0) {
            o.w_tested[out_i] = S.cnt[0];
            o.w_vtests[out_i] = S.cnt[1];
            o.w_cuts[out_i] = S.cnt[2];
            o.w_newv[out_i] = 2 * S.cnt[2];
            o.w_retest[out_i] = S.cnt[3];
            o.w_fallback[out_i] = 0;
            o.w_pref[out_i] = 0;
        }
        __syncwarp(gmask);
    }
}

template <typename T, int G, int CAP, bool BATCH>
cudaError_t launch2_t(const Store &s, const Out &o, const Params &p, const Offsets &off, unsigned *ticket,
                      int sm_count, const int *cells, int ncells, int tier, cudaStream_t st) {
    constexpr int threads = 128;
    const size_t smem = sizeof(Smem2<T, CAP>) * (threads / G);
    auto kfn = k_cells2<T, G, CAP, BATCH>;
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    // the FP64 tiers take few cells: one CTA an SM
    const int grid = (tier > 0 && sizeof(T) == 8) ? sm_count : sm_count * per_sm;
    if ((e = cudaMemsetAsync(ticket, 0, sizeof(unsigned), st)) != cudaSuccess) return e;
    ++g_launch_count;
    kfn<<<grid, threads, smem, st>>>(s, o, p, off, ticket, cells, ncells, tier);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_cells2(const Store &s, const Out &o, const Params &p, const Offsets &off, int precision,
                          unsigned *ticket, int sm_count, int warps_per_cta, const int *cells, int ncells, int tier,
                          cudaStream_t st) {
    (void)warps_per_cta;
    // FP32 with vg_config.split = 1: tier 0 holds 16 vertices a cell (two
    // per lane), fewer registers and slots per lane than 32, and hands the
    // larger cells to an FP32 tier 1 of 32 (the block bound kept: the cells
    // that reach far, as at a cluster's surface, are the ones with many
    // vertices); split = 0: tier 0 holds 32, as the FP64 form.  The rare
    // large cells (tiers 1, 2) always take the batched form.
    const bool small0 = precision != VG_FP64 && p.split;
    if (tier == 2) return launch2_t<double, 32, 64, true>(s, o, p, off, ticket, sm_count, cells, ncells, tier, st);
    if (tier == 1)
        return small0 ? launch2_t<float, 8, 32, true>(s, o, p, off, ticket, sm_count, cells, ncells, tier, st)
                      : launch2_t<double, 16, 64, true>(s, o, p, off, ticket, sm_count, cells, ncells, tier, st);
    const bool batch = s.nsys > 1;
    if (precision == VG_FP64)
        return batch ? launch2_t<double, 8, 32, true>(s, o, p, off, ticket, sm_count, cells, ncells, 0, st)
                     : launch2_t<double, 8, 32, false>(s, o, p, off, ticket, sm_count, cells, ncells, 0, st);
    if (small0)
        return batch ? launch2_t<float, 8, 16, true>(s, o, p, off, ticket, sm_count, cells, ncells, 0, st)
                     : launch2_t<float, 8, 16, false>(s, o, p, off, ticket, sm_count, cells, ncells, 0, st);
    return batch ? launch2_t<float, 8, 32, true>(s, o, p, off, ticket, sm_count, cells, ncells, 0, st)
                 : launch2_t<float, 8, 32, false>(s, o, p, off, ticket, sm_count, cells, ncells, 0, st);
}

}  // namespace vg
