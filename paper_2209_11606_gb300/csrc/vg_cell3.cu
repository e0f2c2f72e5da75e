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
// polyhedron whose vertices are all of degree 3 is stored in its dual form,
// each vertex being the triple of planes (a, b, c) that meet there, ordered
// counter-clockwise seen from outside.  This is the representation used by
// Ray, Sokolov, Lefebvre and Levy, "Meshless Voronoi on the GPU" (ACM TOG
// 2018).  Vertex k lives in lane k % 32, register slot k / 32; its position
// is cached next to its triple.  A cut is:
//   1. classify every vertex against the plane (one FMA chain per lane and
//      slot; a warp ballot tells whether anything is outside);
//   2. mark the directed edges of the removed triangles in a bit matrix;
//      an edge (x, y) of a removed triangle whose twin (y, x) is not marked
//      borders the kept part, and yields the new vertex (x, y, new plane);
//   3. compact kept and new vertices through shared memory with a warp scan.
// FP32 form: positions relative to the particle in FP32; any vertex whose
// signed distance lies within tol32 * R * |q| of the plane is re-solved from
// its three planes in FP64 (from the original FP64 positions) and classified
// there, so the topology follows the FP64 decision; a new vertex whose three
// planes are ill-conditioned is solved in FP64 too.
#include <float.h>

#include "vg_internal.cuh"

namespace vg {
namespace {

constexpr unsigned TRI_EMPTY = 0xffffffffu;
constexpr int KMAX = 128;            // prefetch list capacity
constexpr float KAPPA2 = 0.01f;      // |det|^2 >= KAPPA2 |n1|^2|n2|^2|n3|^2 to stay in FP32
constexpr int MAX_SHELL_EXTRA = 4;

template <typename T> struct V4T;
template <> struct V4T<float> { using t = float4; };
template <> struct __align__(32) V4T<double> { using t = D4; };

template <typename T> __device__ __forceinline__ typename V4T<T>::t mk4(T x, T y, T z, T w);
template <> __device__ __forceinline__ float4 mk4<float>(float x, float y, float z, float w) {
    return make_float4(x, y, z, w);
}
template <> __device__ __forceinline__ D4 mk4<double>(double x, double y, double z, double w) {
    D4 r; r.x = x; r.y = y; r.z = z; r.w = w;
    return r;
}

template <typename T, int VPL, int MAXP>
struct Smem {
    typename V4T<T>::t pl[MAXP];   // plane normal (x,y,z) and constant (w)
    int pref[MAXP];                // neighbour's sorted index, or wall code -1..-6
    int pimg[MAXP];                // packed image shift of the neighbour
    unsigned stri[32 * VPL];       // staging for compaction / statistics
    T sx[32 * VPL], sy[32 * VPL], sz[32 * VPL];
    union {
        unsigned long long E[MAXP][MAXP / 64];  // removed directed edges of one cut
        double dpos[32 * VPL][3];               // FP64 vertices (degenerate cells)
    } u;
    unsigned char ftab[32][MAXP];  // per-lane face walk table
    unsigned long long ckey[KMAX];  // prefetch keys, then face sort keys
};

__device__ __forceinline__ int imgc(int img, int a) { return (int)(signed char)((img >> (8 * a)) & 0xff); }
__device__ __forceinline__ int pack_img(int mx, int my, int mz) {
    return (mx & 0xff) | ((my & 0xff) << 8) | ((mz & 0xff) << 16);
}
__device__ __forceinline__ int floordiv(int a, int b) {
    int q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) q--;
    return q;
}
__device__ __forceinline__ int tri_a(unsigned t) { return t & 0xff; }
__device__ __forceinline__ int tri_b(unsigned t) { return (t >> 8) & 0xff; }
__device__ __forceinline__ int tri_c(unsigned t) { return (t >> 16) & 0xff; }
__device__ __forceinline__ unsigned mk_tri(int a, int b, int c) {
    return (unsigned)a | ((unsigned)b << 8) | ((unsigned)c << 16);
}

__device__ __forceinline__ int warp_excl_scan(int v, int lane, int &total) {
    int x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int y = __shfl_up_sync(FULL, x, d);
        if (lane >= d) x += y;
    }
    total = __shfl_sync(FULL, x, 31);
    return x - v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(FULL, v, d);
    return v;
}
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(FULL, v, d);
    return v;
}
__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v = fmax(v, __shfl_xor_sync(FULL, v, d));
    return v;
}
__device__ __forceinline__ float warp_max_f(float v) {
    // non-negative floats order like their bit patterns
    return __int_as_float((int)__reduce_max_sync(FULL, (unsigned)__float_as_int(v)));
}
__device__ __forceinline__ unsigned long long warp_or64(unsigned long long v) {
    unsigned lo = __reduce_or_sync(FULL, (unsigned)v);
    unsigned hi = __reduce_or_sync(FULL, (unsigned)(v >> 32));
    return ((unsigned long long)hi << 32) | lo;
}

// Per-cell constants.
struct CellIn {
    int i;            // sorted index
    int self_id;      // input index
    int b[3];         // home block
    float o[3];       // FP32 offset inside the home block
    double p[3];      // FP64 position
    double rp;        // radius (radical) or 0
    float rp32;
};

// FP64 plane of a neighbour (sorted index `ref`, image `img`) or of a wall
// (ref = -(1 + 2 axis + side)): the cell lies on n.r <= c, relative to p.
// Same operation order as the oracle's: q = (x_j + m L) - x_p.
__device__ __forceinline__ void plane64(const Grid &g, const Store &s, const CellIn &ci, int ref,
                                        int img, double n[3], double &c) {
    if (ref < 0) {
        int w = -ref - 1, a = w >> 1, side = w & 1;
        n[0] = n[1] = n[2] = 0.0;
        n[a] = side ? 1.0 : -1.0;
        c = side ? __dsub_rn(g.hi[a], ci.p[a]) : __dsub_rn(ci.p[a], g.lo[a]);
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

template <typename T, int VPL, int MAXP>
struct Cell {
    static constexpr int CAP = 32 * VPL;
    static constexpr int NW = MAXP / 64;
    static constexpr bool F32 = sizeof(T) == 4;
    using S_t = Smem<T, VPL, MAXP>;

    S_t &S;
    const Grid &g;
    const Store &st;
    const Params &pp;
    CellIn ci;
    int lane;
    unsigned tri[VPL];
    T vx[VPL], vy[VPL], vz[VPL];
    int ntri;
    unsigned long long live[NW];
    T r2;
    bool degen;
    bool fail;      // capacity or consistency failure: retry on the next tier
    bool empty;
    bool dup;
    double tau64_rel;
    int n_tested, n_vtests, n_cuts, n_retest;

    __device__ Cell(S_t &S_, const Grid &g_, const Store &st_, const Params &pp_, int lane_)
        : S(S_), g(g_), st(st_), pp(pp_), lane(lane_) {}

    // ---- initial cell, Eqs. (1)-(2) ----------------------------------------
    __device__ void init() {
        double lo[3], hi[3];
        for (int a = 0; a < 3; a++) {
            if (g.per[a]) { lo[a] = -0.5 * g.L[a]; hi[a] = 0.5 * g.L[a]; }
            else { lo[a] = __dsub_rn(g.lo[a], ci.p[a]); hi[a] = __dsub_rn(g.hi[a], ci.p[a]); }
        }
        if (lane < 6) {
            int a = lane >> 1, side = lane & 1;
            T n[3] = {0, 0, 0};
            T c;
            int ref, img;
            if (g.per[a]) {
                n[a] = side ? (T)g.L[a] : -(T)g.L[a];
                c = (T)(0.5 * g.L[a] * g.L[a]);
                ref = ci.i;
                int m[3] = {0, 0, 0};
                m[a] = side ? 1 : -1;
                img = pack_img(m[0], m[1], m[2]);
            } else {
                n[a] = side ? (T)1 : (T)-1;
                c = side ? (T)hi[a] : (T)(-lo[a]);
                ref = -(1 + 2 * a + side);
                img = 0;
            }
            S.pl[lane] = mk4<T>(n[0], n[1], n[2], c);
            S.pref[lane] = ref;
            S.pimg[lane] = img;
        }
#pragma unroll
        for (int s = 0; s < VPL; s++) tri[s] = TRI_EMPTY;
        if (lane < 8) {
            int sx = lane & 1, sy = (lane >> 1) & 1, sz = (lane >> 2) & 1;
            int minus = (1 - sx) + (1 - sy) + (1 - sz);
            int A = sx, B = 2 + sy, C = 4 + sz;
            tri[0] = (minus & 1) ? mk_tri(A, C, B) : mk_tri(A, B, C);
            vx[0] = (T)(sx ? hi[0] : lo[0]);
            vy[0] = (T)(sy ? hi[1] : lo[1]);
            vz[0] = (T)(sz ? hi[2] : lo[2]);
        } else {
            vx[0] = vy[0] = vz[0] = (T)0;
        }
#pragma unroll
        for (int s = 1; s < VPL; s++) vx[s] = vy[s] = vz[s] = (T)0;
        ntri = 8;
#pragma unroll
        for (int w = 0; w < NW; w++) live[w] = w == 0 ? 0x3full : 0ull;
        T rr = lane < 8 ? vx[0] * vx[0] + vy[0] * vy[0] + vz[0] * vz[0] : (T)0;
        r2 = warp_max(rr);
        degen = fail = empty = dup = false;
        n_tested = n_vtests = n_cuts = n_retest = 0;
        __syncwarp();
    }

    __device__ __forceinline__ T warp_max(T v) {
        if constexpr (F32) return warp_max_f(v);
        else return warp_max_d(v);
    }

    // FP64 position of the vertex with triple t.
    __device__ void vertex64(unsigned t, double v[3]) {
        double n1[3], n2[3], n3[3], c1, c2, c3;
        int a = tri_a(t), b = tri_b(t), c = tri_c(t);
        plane64(g, st, ci, S.pref[a], S.pimg[a], n1, c1);
        plane64(g, st, ci, S.pref[b], S.pimg[b], n2, c2);
        plane64(g, st, ci, S.pref[c], S.pimg[c], n3, c3);
        solve3_d(n1, c1, n2, c2, n3, c3, v);
    }

    // Position of the new vertex where planes x, y and the cutting plane meet.
    __device__ void new_vertex(int x, int y, T qx, T qy, T qz, T c, int ref, int img, T &ox, T &oy,
                               T &oz) {
        auto P1 = S.pl[x];
        auto P2 = S.pl[y];
        T x23x = P2.y * qz - P2.z * qy, x23y = P2.z * qx - P2.x * qz, x23z = P2.x * qy - P2.y * qx;
        T x31x = qy * P1.z - qz * P1.y, x31y = qz * P1.x - qx * P1.z, x31z = qx * P1.y - qy * P1.x;
        T x12x = P1.y * P2.z - P1.z * P2.y, x12y = P1.z * P2.x - P1.x * P2.z, x12z = P1.x * P2.y - P1.y * P2.x;
        T det = P1.x * x23x + P1.y * x23y + P1.z * x23z;
        if constexpr (F32) {
            T m1 = P1.x * P1.x + P1.y * P1.y + P1.z * P1.z;
            T m2 = P2.x * P2.x + P2.y * P2.y + P2.z * P2.z;
            T m3 = qx * qx + qy * qy + qz * qz;
            if (!(det * det >= KAPPA2 * m1 * m2 * m3)) {
                double n1[3], n2[3], n3[3], c1, c2, c3, v[3];
                plane64(g, st, ci, S.pref[x], S.pimg[x], n1, c1);
                plane64(g, st, ci, S.pref[y], S.pimg[y], n2, c2);
                plane64(g, st, ci, ref, img, n3, c3);
                solve3_d(n1, c1, n2, c2, n3, c3, v);
                ox = (T)v[0]; oy = (T)v[1]; oz = (T)v[2];
                return;
            }
        }
        T id = (T)1 / det;
        ox = (P1.w * x23x + P2.w * x31x + c * x12x) * id;
        oy = (P1.w * x23y + P2.w * x31y + c * x12y) * id;
        oz = (P1.w * x23z + P2.w * x31z + c * x12z) * id;
    }

    // Cut by the plane q.r = c of neighbour (ref, img).  Returns 0 when
    // nothing is removed, 1 when the cell changed, 2 when it became empty,
    // 3 on a capacity failure.
    __device__ int cut(T qx, T qy, T qz, T c, T qq, int ref, int img) {
        n_tested++;
        n_vtests += ntri;
        T tau;
        if constexpr (F32) tau = (T)pp.tol32 * sqrtf(r2 * qq);
        else tau = (T)(tau64_rel * sqrt((double)qq));
        unsigned outm = 0, nearm = 0, onm = 0;
#pragma unroll
        for (int s = 0; s < VPL; s++) {
            if (s * 32 < ntri) {
                bool valid = tri[s] != TRI_EMPTY;
                T d = vx[s] * qx + vy[s] * qy + vz[s] * qz - c;
                if (valid) {
                    if (d > tau) outm |= 1u << s;
                    else if (d >= -tau) {
                        if constexpr (F32) nearm |= 1u << s;
                        else onm |= 1u << s;
                    }
                }
            }
        }
        if constexpr (F32) {
            if (__any_sync(FULL, nearm)) {
                n_retest++;
                double n3[3], c3;
                plane64(g, st, ci, ref, img, n3, c3);
                double qn = sqrt(n3[0] * n3[0] + n3[1] * n3[1] + n3[2] * n3[2]);
                double tau64 = tau64_rel * qn;
#pragma unroll
                for (int s = 0; s < VPL; s++) {
                    if (nearm & (1u << s)) {
                        double v[3];
                        vertex64(tri[s], v);
                        double d = __dsub_rn(__dadd_rn(__dadd_rn(__dmul_rn(n3[0], v[0]), __dmul_rn(n3[1], v[1])),
                                                       __dmul_rn(n3[2], v[2])),
                                             c3);
                        if (d > tau64) outm |= 1u << s;
                        else if (d >= -tau64) onm |= 1u << s;
                    }
                }
            }
        }
        if (!__any_sync(FULL, outm)) return 0;
        if (__any_sync(FULL, onm)) degen = true;
        n_cuts++;
        // free plane slot
        int np = -1;
#pragma unroll
        for (int w = NW - 1; w >= 0; w--)
            if (~live[w]) np = w * 64 + __ffsll((long long)~live[w]) - 1;
        if (np < 0) return 3;
        // mark the directed edges of removed triangles
#pragma unroll
        for (int s = 0; s < VPL; s++) {
            if (outm & (1u << s)) {
                int a = tri_a(tri[s]), b = tri_b(tri[s]), cc = tri_c(tri[s]);
                atomicOr(&S.u.E[a][b >> 6], 1ull << (b & 63));
                atomicOr(&S.u.E[b][cc >> 6], 1ull << (cc & 63));
                atomicOr(&S.u.E[cc][a >> 6], 1ull << (a & 63));
            }
        }
        __syncwarp();
        unsigned bnd[VPL];
        int cnt = 0;
#pragma unroll
        for (int s = 0; s < VPL; s++) {
            bnd[s] = 0;
            if (outm & (1u << s)) {
                int a = tri_a(tri[s]), b = tri_b(tri[s]), cc = tri_c(tri[s]);
                // edge (x,y) borders the kept part iff its twin (y,x) was not removed
                if (!((S.u.E[b][a >> 6] >> (a & 63)) & 1)) bnd[s] |= 1;
                if (!((S.u.E[cc][b >> 6] >> (b & 63)) & 1)) bnd[s] |= 2;
                if (!((S.u.E[a][cc >> 6] >> (cc & 63)) & 1)) bnd[s] |= 4;
                cnt += __popc(bnd[s]);
            } else if (tri[s] != TRI_EMPTY) {
                cnt++;
            }
        }
        int total;
        int base = warp_excl_scan(cnt, lane, total);
        int rc = 1;
        if (total > CAP) rc = 3;
        else if (total == 0) rc = 2;
        if (rc == 1) {
            // write kept and new vertices to staging
#pragma unroll
            for (int s = 0; s < VPL; s++) {
                if (outm & (1u << s)) {
                    int a = tri_a(tri[s]), b = tri_b(tri[s]), cc = tri_c(tri[s]);
                    int ex[3] = {a, b, cc}, ey[3] = {b, cc, a};
#pragma unroll
                    for (int e = 0; e < 3; e++) {
                        if (bnd[s] & (1u << e)) {
                            T ox, oy, oz;
                            new_vertex(ex[e], ey[e], qx, qy, qz, c, ref, img, ox, oy, oz);
                            S.stri[base] = mk_tri(ex[e], ey[e], np);
                            S.sx[base] = ox; S.sy[base] = oy; S.sz[base] = oz;
                            base++;
                        }
                    }
                } else if (tri[s] != TRI_EMPTY) {
                    S.stri[base] = tri[s];
                    S.sx[base] = vx[s]; S.sy[base] = vy[s]; S.sz[base] = vz[s];
                    base++;
                }
            }
        }
        __syncwarp();
        // clear the marked rows
#pragma unroll
        for (int s = 0; s < VPL; s++) {
            if (outm & (1u << s)) {
                int a = tri_a(tri[s]), b = tri_b(tri[s]), cc = tri_c(tri[s]);
#pragma unroll
                for (int w = 0; w < NW; w++) { S.u.E[a][w] = 0; S.u.E[b][w] = 0; S.u.E[cc][w] = 0; }
            }
        }
        if (rc != 1) { __syncwarp(); return rc; }
        if (lane == 0) {
            S.pl[np] = mk4<T>(qx, qy, qz, c);
            S.pref[np] = ref;
            S.pimg[np] = img;
        }
        __syncwarp();
        ntri = total;
        unsigned long long lv[NW];
#pragma unroll
        for (int w = 0; w < NW; w++) lv[w] = 0;
        T rr = 0;
#pragma unroll
        for (int s = 0; s < VPL; s++) {
            int t = s * 32 + lane;
            if (t < total) {
                tri[s] = S.stri[t];
                vx[s] = S.sx[t]; vy[s] = S.sy[t]; vz[s] = S.sz[t];
                int a = tri_a(tri[s]), b = tri_b(tri[s]), cc = tri_c(tri[s]);
                lv[a >> 6] |= 1ull << (a & 63);
                lv[b >> 6] |= 1ull << (b & 63);
                lv[cc >> 6] |= 1ull << (cc & 63);
                T q2 = vx[s] * vx[s] + vy[s] * vy[s] + vz[s] * vz[s];
                rr = rr > q2 ? rr : q2;
            } else {
                tri[s] = TRI_EMPTY;
            }
        }
#pragma unroll
        for (int w = 0; w < NW; w++) live[w] = warp_or64(lv[w]);
        r2 = warp_max(rr);
        __syncwarp();
        return 1;
    }

    // Radius bound (Sec. 2.1.3), squared, with a small relative margin that
    // covers the rounding of R and of candidate distances.
    __device__ __forceinline__ T stop2() {
        T margin = F32 ? (T)1.0001 : (T)(1.0 + 1e-12);
        if (!st.radical) return (T)4 * r2 * margin;
        T R = sqrt(r2);
        T disc = r2 + (T)(st.rmax * st.rmax) - (T)(ci.rp * ci.rp);
        if (disc <= (T)0) return (T)0;
        T rs = R + sqrt(disc);
        return rs * rs * margin;
    }
};

// ---- candidate generation ----------------------------------------------------

// FP32 relative position of particle pj seen from the cell's particle through
// block offset (ox, oy, oz); used identically by the prefetch gather and the
// walk so that both see bit-identical distances.
__device__ __forceinline__ void cand32(const Grid &g, const CellIn &ci, float4 pj, int ox, int oy,
                                       int oz, float &qx, float &qy, float &qz, float &qq) {
    qx = __fadd_rn(__fmul_rn((float)ox, g.hf[0]), __fsub_rn(pj.x, ci.o[0]));
    qy = __fadd_rn(__fmul_rn((float)oy, g.hf[1]), __fsub_rn(pj.y, ci.o[1]));
    qz = __fadd_rn(__fmul_rn((float)oz, g.hf[2]), __fsub_rn(pj.z, ci.o[2]));
    qq = __fadd_rn(__fadd_rn(__fmul_rn(qx, qx), __fmul_rn(qy, qy)), __fmul_rn(qz, qz));
}

__device__ __forceinline__ void cand64(const Grid &g, const CellIn &ci, D4 pj, int mx, int my, int mz,
                                       double &qx, double &qy, double &qz, double &qq) {
    qx = __dsub_rn(__dadd_rn(pj.x, __dmul_rn((double)mx, g.L[0])), ci.p[0]);
    qy = __dsub_rn(__dadd_rn(pj.y, __dmul_rn((double)my, g.L[1])), ci.p[1]);
    qz = __dsub_rn(__dadd_rn(pj.z, __dmul_rn((double)mz, g.L[2])), ci.p[2]);
    qq = __dadd_rn(__dadd_rn(__dmul_rn(qx, qx), __dmul_rn(qy, qy)), __dmul_rn(qz, qz));
}

// Squared distance from the particle to the box of the block at offset o
// (block-relative), FP32.
__device__ __forceinline__ float block_gap2(const Grid &g, const CellIn &ci, int ox, int oy, int oz) {
    int o[3] = {ox, oy, oz};
    float d2 = 0.f;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        float lo = (float)o[a] * g.hf[a] - ci.o[a];
        float hi = lo + g.hf[a];
        float gap = lo > 0.f ? lo : (hi < 0.f ? -hi : 0.f);
        d2 += gap * gap;
    }
    return d2;
}

// Resolves block offset o: returns false if it falls outside a walled box;
// otherwise the linear block index and the image shift.
__device__ __forceinline__ bool resolve(const Grid &g, const CellIn &ci, const int o[3], int &k, int m[3]) {
    int t[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        int ta = ci.b[a] + o[a];
        m[a] = 0;
        if (g.per[a]) {
            m[a] = floordiv(ta, g.nb[a]);
            ta -= m[a] * g.nb[a];
        } else if (ta < 0 || ta >= g.nb[a]) {
            return false;
        }
        t[a] = ta;
    }
    k = t[0] + g.nb[0] * (t[1] + g.nb[1] * t[2]);
    return true;
}

template <typename T, int VPL, int MAXP>
struct Driver {
    using C_t = Cell<T, VPL, MAXP>;
    static constexpr bool F32 = C_t::F32;

    // Offer every particle of the block at offset o (if not skipped) to the
    // cell.  skip_rho2 > 0: skip particles with o inside the prefetch box and
    // FP32 distance^2 < skip_rho2 (already cut by the prefetch pass).
    // Returns false if the cell ended (empty or failure).
    static __device__ bool offer_block(C_t &C, const Grid &g, const Store &st, const int o[3],
                                       T &stop, float skip_rho2, const int *rg) {
        int k, m[3];
        if (!resolve(g, C.ci, o, k, m)) return true;
        float gap2 = block_gap2(g, C.ci, o[0], o[1], o[2]);
        if ((T)gap2 * (T)0.99998 >= stop) return true;
        // particles the prefetch pass already offered: inside its block box,
        // in a block it gathered, and closer than its radius
        bool in_pref = skip_rho2 > 0.f && abs(o[0]) <= rg[0] && abs(o[1]) <= rg[1] &&
                       abs(o[2]) <= rg[2] && gap2 < skip_rho2;
        int j0 = __ldg(&st.bstart[k]), j1 = __ldg(&st.bstart[k + 1]);
        int img = pack_img(m[0], m[1], m[2]);
        bool self_block = (o[0] == 0 && o[1] == 0 && o[2] == 0);
        for (int base = j0; base < j1; base += 32) {
            int j = base + C.lane;
            T qx = 0, qy = 0, qz = 0, qq = 0, rj = 0;
            bool ok = j < j1;
            if (ok) {
                if constexpr (F32) {
                    float4 pj = __ldg(&st.p32[j]);
                    cand32(g, C.ci, pj, o[0], o[1], o[2], qx, qy, qz, qq);
                    rj = pj.w;
                    if (in_pref && qq < skip_rho2) ok = false;
                } else {
                    D4 pj = st.p64[j];
                    cand64(g, C.ci, pj, m[0], m[1], m[2], qx, qy, qz, qq);
                    rj = pj.w;
                }
                if (self_block && j == C.ci.i) ok = false;
            }
            unsigned want = __ballot_sync(FULL, ok);
            while (want) {
                int src = __ffs(want) - 1;
                want &= want - 1;
                T bx = __shfl_sync(FULL, qx, src), by = __shfl_sync(FULL, qy, src);
                T bz = __shfl_sync(FULL, qz, src), bq = __shfl_sync(FULL, qq, src);
                T br = __shfl_sync(FULL, rj, src);
                if (bq >= stop) continue;
                if (bq < (T)1e-30) { C.dup = true; continue; }
                T c = (T)0.5 * (bq + (T)(C.ci.rp32 * C.ci.rp32) - br * br);
                if constexpr (!F32) c = 0.5 * (bq + C.ci.rp * C.ci.rp - br * br);
                int r = C.cut(bx, by, bz, c, bq, base + src, img);
                if (r == 2) { C.empty = true; return false; }
                if (r == 3) { C.fail = true; return false; }
                if (r == 1) stop = C.stop2();
            }
        }
        return true;
    }

    // The walk of Sec. 2.1.3: blocks in ascending order of their distance
    // bound from the home block, stopped by the radius bound.
    static __device__ bool walk(C_t &C, const Grid &g, const Store &st, const Offsets &off,
                                float skip_rho2, const int *rg, int &limit_hit) {
        T stop = C.stop2();
        int e = 0;
        for (; e < off.count; e++) {
            float lb = __ldg(&off.lb[e]);
            if ((T)(lb * lb) * (T)0.99998 >= stop) break;
            int code = __ldg(&off.code[e]);
            int o[3] = {imgc(code, 0), imgc(code, 1), imgc(code, 2)};
            if (!offer_block(C, g, st, o, stop, skip_rho2, rg)) return false;
        }
        if (e < off.count) return true;
        // beyond the list: Chebyshev shells, skipping offsets the list held
        float hmin = fminf(g.hf[0], fminf(g.hf[1], g.hf[2]));
        float lbmax = (float)off.shell * hmin;
        int maxs = off.shell + MAX_SHELL_EXTRA + 2 * max(g.nb[0], max(g.nb[1], g.nb[2]));
        for (int s = 1; s <= maxs; s++) {
            float sb = (float)(s - 1) * hmin;
            if ((T)(sb * sb) * (T)0.99998 >= stop) return true;
            for (int ox = -s; ox <= s; ox++)
                for (int oy = -s; oy <= s; oy++)
                    for (int oz = -s; oz <= s; oz++) {
                        if (max(abs(ox), max(abs(oy), abs(oz))) != s) continue;
                        float lbx = fmaxf(0.f, (float)(abs(ox) - 1)) * g.hf[0];
                        float lby = fmaxf(0.f, (float)(abs(oy) - 1)) * g.hf[1];
                        float lbz = fmaxf(0.f, (float)(abs(oz) - 1)) * g.hf[2];
                        float lb2 = lbx * lbx + lby * lby + lbz * lbz;
                        if (lb2 < lbmax * lbmax) continue;  // held by the list
                        int o[3] = {ox, oy, oz};
                        if (!offer_block(C, g, st, o, stop, skip_rho2, rg)) return false;
                    }
        }
        limit_hit = 1;
        return true;
    }
};

// Bitonic sort of 32*E keys held E per lane (element g = lane*E + e).
template <int E>
__device__ __forceinline__ void bitonic(unsigned long long (&k)[E], int lane) {
#pragma unroll
    for (int size = 2; size <= 32 * E; size <<= 1) {
#pragma unroll
        for (int j = size >> 1; j > 0; j >>= 1) {
            if (j < E) {
#pragma unroll
                for (int e = 0; e < E; e++) {
                    if ((e & j) == 0) {
                        int gi = lane * E + e;
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
                    int gi = lane * E + e;
                    bool up = (gi & size) == 0;
                    unsigned long long o = __shfl_xor_sync(FULL, k[e], lm);
                    bool lower = (gi & j) == 0;
                    bool keep_min = (lower == up);
                    unsigned long long mn = k[e] < o ? k[e] : o, mx = k[e] < o ? o : k[e];
                    k[e] = keep_min ? mn : mx;
                }
            }
        }
    }
}

// ---- statistics ----------------------------------------------------------------

template <typename T, int VPL, int MAXP>
__device__ void finish(Cell<T, VPL, MAXP> &C, const Out &o, const Grid &g, const Store &st,
                       const Params &pp, int status) {
    using C_t = Cell<T, VPL, MAXP>;
    constexpr int NW = C_t::NW;
    auto &S = C.S;
    const int lane = C.lane;
    const int out_i = C.ci.self_id;
    if (status != VG_CELL_OK) {
        if (lane == 0) {
            o.vol[out_i] = 0; o.area[out_i] = 0;
            for (int a = 0; a < 3; a++) o.cen[(long long)out_i * 3 + a] = 0;
            o.nv[out_i] = 0; o.ne[out_i] = 0; o.nf[out_i] = 0;
            o.status[out_i] = (unsigned char)status;
            o.fptr[out_i] = 0;
        }
        return;
    }
    // stage vertices
    const int T_ = C.ntri;
#pragma unroll
    for (int s = 0; s < VPL; s++) {
        int t = s * 32 + lane;
        if (t < T_) { S.stri[t] = C.tri[s]; S.sx[t] = C.vx[s]; S.sy[t] = C.vy[s]; S.sz[t] = C.vz[s]; }
    }
    double eps = pp.merge_rel * g.s;
    double eps2 = eps * eps;
    if (C.degen) {
#pragma unroll
        for (int s = 0; s < VPL; s++) {
            int t = s * 32 + lane;
            if (t < T_) {
                double v[3];
                if constexpr (C_t::F32) C.vertex64(C.tri[s], v);
                else { v[0] = C.vx[s]; v[1] = C.vy[s]; v[2] = C.vz[s]; }
                S.u.dpos[t][0] = v[0]; S.u.dpos[t][1] = v[1]; S.u.dpos[t][2] = v[2];
            }
        }
    }
    __syncwarp();
    // live planes -> faces; lane handles face f = lane, lane + 32, ...
    int F = 0;
#pragma unroll
    for (int w = 0; w < NW; w++) F += __popcll(C.live[w]);
    double vol = 0, area = 0, cx = 0, cy = 0, cz = 0;
    int order_sum = 0, faces_kept = 0;
    bool bad = false;
    constexpr int R = MAXP / 32;
    unsigned long long key[R];
    int fn[R], fi[R], fo[R];
#pragma unroll
    for (int r = 0; r < R; r++) { key[r] = ~0ull; fn[r] = fi[r] = fo[r] = 0; }
    for (int rnd = 0; rnd * 32 < F; rnd++) {
        int f = rnd * 32 + lane;
        // the f-th live plane
        int a = -1;
        if (f < F) {
            int cntw = 0;
            for (int w = 0; w < NW; w++) {
                int pc = __popcll(C.live[w]);
                if (f < cntw + pc) {
                    unsigned long long m = C.live[w];
                    int r = f - cntw;
                    for (int u = 0; u < r; u++) m &= m - 1;
                    a = w * 64 + __ffsll((long long)m) - 1;
                    break;
                }
                cntw += pc;
            }
        }
        int t0 = -1, deg = 0;
        for (int t = 0; t < T_; t++) {
            unsigned tr = S.stri[t];
            if (a >= 0) {
                int p0 = tri_a(tr), p1 = tri_b(tr), p2 = tri_c(tr);
                int xx = -1;
                if (p0 == a) xx = p1;
                else if (p1 == a) xx = p2;
                else if (p2 == a) xx = p0;
                if (xx >= 0) {
                    S.ftab[lane][xx] = (unsigned char)t;
                    if (t0 < 0) t0 = t;
                    deg++;
                }
            }
        }
        __syncwarp();
        if (a >= 0) {
            if (deg < 3) bad = true;
            // walk the face counter-clockwise from outside
            int cur = t0;
            double fvol = 0, fcx = 0, fcy = 0, fcz = 0, fax = 0, fay = 0, faz = 0, per = 0;
            int distinct = 0;
            T u0x = S.sx[t0], u0y = S.sy[t0], u0z = S.sz[t0];
            int steps = 0;
            double px = 0, py = 0, pz = 0;  // FP64 previous distinct point (degenerate cells)
            double fx = 0, fy = 0, fz = 0;
            if (C.degen) { fx = S.u.dpos[t0][0]; fy = S.u.dpos[t0][1]; fz = S.u.dpos[t0][2]; px = fx; py = fy; pz = fz; distinct = 1; }
            for (steps = 0; steps < deg; steps++) {
                unsigned tr = S.stri[cur];
                int p0 = tri_a(tr), p1 = tri_b(tr), p2 = tri_c(tr);
                int yy;
                if (p0 == a) yy = p2;
                else if (p1 == a) yy = p0;
                else if (p2 == a) yy = p1;
                else { bad = true; break; }
                int nx = S.ftab[lane][yy];
                if (nx >= T_) { bad = true; break; }
                if (nx == t0) { steps++; break; }
                if (cur != t0) {
                    if (C.degen) {
                        double ax = S.u.dpos[cur][0] - fx, ay = S.u.dpos[cur][1] - fy, az = S.u.dpos[cur][2] - fz;
                        double bx2 = S.u.dpos[nx][0] - fx, by2 = S.u.dpos[nx][1] - fy, bz2 = S.u.dpos[nx][2] - fz;
                        double det = fx * (S.u.dpos[cur][1] * S.u.dpos[nx][2] - S.u.dpos[cur][2] * S.u.dpos[nx][1]) -
                                     fy * (S.u.dpos[cur][0] * S.u.dpos[nx][2] - S.u.dpos[cur][2] * S.u.dpos[nx][0]) +
                                     fz * (S.u.dpos[cur][0] * S.u.dpos[nx][1] - S.u.dpos[cur][1] * S.u.dpos[nx][0]);
                        fvol += det;
                        fcx += det * (fx + S.u.dpos[cur][0] + S.u.dpos[nx][0]);
                        fcy += det * (fy + S.u.dpos[cur][1] + S.u.dpos[nx][1]);
                        fcz += det * (fz + S.u.dpos[cur][2] + S.u.dpos[nx][2]);
                        fax += ay * bz2 - az * by2;
                        fay += az * bx2 - ax * bz2;
                        faz += ax * by2 - ay * bx2;
                    } else {
                        T ax = S.sx[cur], ay = S.sy[cur], az = S.sz[cur];
                        T bx2 = S.sx[nx], by2 = S.sy[nx], bz2 = S.sz[nx];
                        T det = u0x * (ay * bz2 - az * by2) - u0y * (ax * bz2 - az * bx2) + u0z * (ax * by2 - ay * bx2);
                        fvol += (double)det;
                        fcx += (double)(det * (u0x + ax + bx2));
                        fcy += (double)(det * (u0y + ay + by2));
                        fcz += (double)(det * (u0z + az + bz2));
                        T e1x = ax - u0x, e1y = ay - u0y, e1z = az - u0z;
                        T e2x = bx2 - u0x, e2y = by2 - u0y, e2z = bz2 - u0z;
                        fax += (double)(e1y * e2z - e1z * e2y);
                        fay += (double)(e1z * e2x - e1x * e2z);
                        faz += (double)(e1x * e2y - e1y * e2x);
                    }
                }
                if (C.degen) {
                    double dx = S.u.dpos[nx][0] - px, dy = S.u.dpos[nx][1] - py, dz = S.u.dpos[nx][2] - pz;
                    if (dx * dx + dy * dy + dz * dz > eps2) {
                        per += sqrt(dx * dx + dy * dy + dz * dz);
                        distinct++;
                        px = S.u.dpos[nx][0]; py = S.u.dpos[nx][1]; pz = S.u.dpos[nx][2];
                    }
                }
                cur = nx;
            }
            if (steps != deg) bad = true;
            double farea = 0.5 * sqrt(fax * fax + fay * fay + faz * faz);
            int order = deg;
            bool keep = true;
            if (C.degen) {
                // close the polygon back to its first point
                double dx = fx - px, dy = fy - py, dz = fz - pz;
                if (distinct > 1 && dx * dx + dy * dy + dz * dz <= eps2) distinct--;
                else per += sqrt(dx * dx + dy * dy + dz * dz);
                order = distinct;
                keep = distinct >= 3 && farea > eps * per;
            }
            vol += fvol;
            cx += fcx; cy += fcy; cz += fcz;
            if (keep) {
                area += farea;
                order_sum += order;
                faces_kept++;
                int ref = S.pref[a];
                int nid = ref >= 0 ? __ldg(&st.sid[ref]) : ref;
                int img = S.pimg[a];
                unsigned ib = ((unsigned)(imgc(img, 0) + 128) << 16) | ((unsigned)(imgc(img, 1) + 128) << 8) |
                              (unsigned)(imgc(img, 2) + 128);
                // canonical order: ascending neighbour id (walls first), then image
#pragma unroll
                for (int r = 0; r < R; r++)
                    if (r == rnd) {
                        key[r] = ((unsigned long long)((long long)nid + 8) << 24) | ib;
                        fn[r] = nid;
                        fi[r] = img & 0xffffff;
                        fo[r] = order;
                    }
            }
        }
        __syncwarp();
    }
    // reductions
    vol = warp_sum_d(vol);
    cx = warp_sum_d(cx); cy = warp_sum_d(cy); cz = warp_sum_d(cz);
    area = warp_sum_d(area);
    int nfk = __reduce_add_sync(FULL, faces_kept);
    int osum = __reduce_add_sync(FULL, order_sum);
    bool anybad = __any_sync(FULL, bad);
    int nv;
    if (C.degen) {
        // distinct vertices: a vertex counts if no earlier vertex coincides
        int cnt = 0;
        for (int s = 0; s < VPL; s++) {
            int t = s * 32 + lane;
            if (t < T_) {
                bool first = true;
                for (int u = 0; u < t && first; u++) {
                    double dx = S.u.dpos[u][0] - S.u.dpos[t][0], dy = S.u.dpos[u][1] - S.u.dpos[t][1],
                           dz = S.u.dpos[u][2] - S.u.dpos[t][2];
                    if (dx * dx + dy * dy + dz * dz <= eps2) first = false;
                }
                cnt += first;
            }
        }
        nv = __reduce_add_sync(FULL, cnt);
    } else {
        nv = T_;
        if (nfk != T_ / 2 + 2) anybad = true;  // Euler: V - 3V/2 + F = 2
    }
    if (anybad) {
        // inconsistent topology: hand the cell to the FP64 big-cell tier
        C.fail = true;
        return;
    }
    // canonical face order by ranking the (unique) keys
#pragma unroll
    for (int r = 0; r < R; r++) S.ckey[r * 32 + lane] = key[r];
    __syncwarp();
    const int cnt_out = nfk;
    long long fbase = 0;
    if (lane == 0) fbase = (long long)atomicAdd(o.fcount, (unsigned long long)cnt_out);
    fbase = __shfl_sync(FULL, fbase, 0);
    const bool overflow = fbase + cnt_out > o.fcap;
#pragma unroll
    for (int r = 0; r < R; r++) {
        if (key[r] != ~0ull && !overflow) {
            int rank = 0;
            for (int u = 0; u < MAXP; u++) rank += S.ckey[u] < key[r];
            int2 ent;
            ent.x = fn[r];
            ent.y = fi[r] | (fo[r] << 24);
            o.faces[fbase + rank] = ent;
        }
    }
    __syncwarp();
    if (lane == 0) {
        o.vol[out_i] = vol / 6.0;
        o.area[out_i] = area;
        double v6 = vol;
        o.cen[(long long)out_i * 3 + 0] = v6 != 0 ? cx / (4.0 * v6) : 0.0;
        o.cen[(long long)out_i * 3 + 1] = v6 != 0 ? cy / (4.0 * v6) : 0.0;
        o.cen[(long long)out_i * 3 + 2] = v6 != 0 ? cz / (4.0 * v6) : 0.0;
        o.nv[out_i] = nv;
        o.ne[out_i] = osum / 2;
        o.nf[out_i] = nfk;
        o.status[out_i] = overflow ? (unsigned char)VG_CELL_CAP : (unsigned char)VG_CELL_OK;
        o.fptr[out_i] = fbase;
    }
}

// ---- the kernel ----------------------------------------------------------------

template <typename T, int VPL, int MAXP>
__global__ void __launch_bounds__(256) k_cells3(Grid g, Store st, Out o, Params pp, Offsets off,
                                                unsigned *ticket, const int *cells, int ncells,
                                                int tier) {
    using C_t = Cell<T, VPL, MAXP>;
    using S_t = Smem<T, VPL, MAXP>;
    extern __shared__ __align__(32) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    S_t &S = reinterpret_cast<S_t *>(smem_raw)[warp];
    // clear the edge matrix once; every cut leaves it clear
    for (int u = lane; u < MAXP * (MAXP / 64); u += 32) (&S.u.E[0][0])[u] = 0ull;
    __syncwarp();
    const int total = cells ? (tier > 0 ? *o.retry_count : ncells) : st.n;
    const int chunk = pp.chunk > 0 ? pp.chunk : 1;
    C_t C(S, g, st, pp, lane);
    C.tau64_rel = pp.tau_rel * g.s;
    for (int iter = 0; iter < (1 << 30); iter++) {
        int base = 0;
        if (lane == 0) base = (int)atomicAdd(ticket, (unsigned)chunk);
        base = __shfl_sync(FULL, base, 0);
        if (base >= total) break;
        int end = min(base + chunk, total);
        for (int w = base; w < end; w++) {
            int i = cells ? cells[w] : w;
            // cell setup
            CellIn &ci = C.ci;
            ci.i = i;
            ci.self_id = __ldg(&st.sid[i]);
            int k = __ldg(&st.sblk[i]);
            ci.b[0] = k % g.nb[0];
            ci.b[1] = (k / g.nb[0]) % g.nb[1];
            ci.b[2] = k / (g.nb[0] * g.nb[1]);
            float4 p32 = __ldg(&st.p32[i]);
            D4 p64 = st.p64[i];
            ci.o[0] = p32.x; ci.o[1] = p32.y; ci.o[2] = p32.z;
            ci.p[0] = p64.x; ci.p[1] = p64.y; ci.p[2] = p64.z;
            ci.rp = p64.w;
            ci.rp32 = p32.w;
            C.init();
            int limit_hit = 0;
            int fell_back = 0;
            bool alive = true;
            int rg[3] = {0, 0, 0};
            float rho2 = 0.f;
            if (pp.order == VG_PREFETCH && C_t::F32 && st.n < (1 << 27)) {
                // ---- prefetch: gather candidates within rho, sort, cut in order
                float kt = (float)(pp.prefetch_k > 0 ? pp.prefetch_k : 72);
                if (pp.kblock) kt = fmaxf(8.f, __ldg(&pp.kblock[k]));
                // local density from the 27 surrounding blocks
                int n27 = 0;
                if (lane < 27) {
                    int o3[3] = {lane % 3 - 1, (lane / 3) % 3 - 1, lane / 9 - 1};
                    int kk, m[3];
                    if (resolve(g, ci, o3, kk, m)) n27 = __ldg(&st.bstart[kk + 1]) - __ldg(&st.bstart[kk]);
                    else n27 = -1000000;  // outside a wall: no volume
                }
                int nin = 0, nvol = 0;
                {
                    int v = n27 >= 0 ? n27 : 0;
                    nin = __reduce_add_sync(FULL, v);
                    nvol = __reduce_add_sync(FULL, (lane < 27 && n27 >= 0) ? 1 : 0);
                }
                float bvol = g.hf[0] * g.hf[1] * g.hf[2];
                float dens = (float)max(nin, 1) / ((float)max(nvol, 1) * bvol);
                float rho = cbrtf(3.f * kt / (4.f * 3.14159265f * dens));
                for (int a = 0; a < 3; a++) rg[a] = min((int)ceilf(rho / g.hf[a]), 63);
                int count = 0;
                for (int attempt = 0; attempt < 6; attempt++) {
                    rho2 = rho * rho;
                    count = 0;
                    for (int oz = -rg[2]; oz <= rg[2]; oz++)
                        for (int oy = -rg[1]; oy <= rg[1]; oy++)
                            for (int ox = -rg[0]; ox <= rg[0]; ox++) {
                                if (block_gap2(g, ci, ox, oy, oz) >= rho2) continue;
                                int o3[3] = {ox, oy, oz}, kk, m[3];
                                if (!resolve(g, ci, o3, kk, m)) continue;
                                int j0 = __ldg(&st.bstart[kk]), j1 = __ldg(&st.bstart[kk + 1]);
                                int oid = (ox + 63) | ((oy + 63) << 7) | ((oz + 63) << 14);
                                for (int b0 = j0; b0 < j1; b0 += 32) {
                                    int j = b0 + lane;
                                    bool keep = false;
                                    float qq = 0.f;
                                    if (j < j1) {
                                        float4 pj = __ldg(&st.p32[j]);
                                        float qx, qy, qz;
                                        cand32(g, ci, pj, ox, oy, oz, qx, qy, qz, qq);
                                        keep = qq < rho2 && !(j == i && ox == 0 && oy == 0 && oz == 0);
                                    }
                                    unsigned bal = __ballot_sync(FULL, keep);
                                    int pos = count + __popc(bal & ((1u << lane) - 1));
                                    if (keep && pos < KMAX) {
                                        // distance^2 bits and the particle; its block offset
                                        // goes to a side table indexed by the same slot
                                        S.ckey[pos] = ((unsigned long long)__float_as_uint(qq) << 32) |
                                                      (unsigned)j;
                                        reinterpret_cast<int *>(S.ftab)[pos] = oid;
                                    }
                                    count += __popc(bal);
                                }
                            }
                    if (count <= KMAX) break;
                    rho *= 0.8f * cbrtf((float)KMAX / (float)count);
                    for (int a = 0; a < 3; a++) rg[a] = min((int)ceilf(rho / g.hf[a]), 63);
                }
                __syncwarp();
                if (count > KMAX) {
                    rho2 = 0.f;  // give up on prefetch: plain walk
                    count = 0;
                }
                // sort the slots by (distance^2, slot): the gather order is
                // deterministic, so equal distances keep a fixed order
                unsigned long long kk4[4];
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    int slot = lane * 4 + e;
                    kk4[e] = slot < count
                                 ? ((S.ckey[slot] & 0xffffffff00000000ull) | (unsigned long long)slot)
                                 : ~0ull;
                }
                bitonic<4>(kk4, lane);
                // sorted slots -> ftab region 2 (after the 128 ints of offset ids)
                int *sorted_slot = reinterpret_cast<int *>(S.ftab) + KMAX;
                __syncwarp();
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    int pos = lane * 4 + e;
                    if (pos < count) sorted_slot[pos] = (int)(kk4[e] & 0xffffffffu);
                }
                __syncwarp();
                // cut in ascending distance
                float stopf = (float)C.stop2();
                int u = 0;
                for (; u < count && alive; u++) {
                    int slot = sorted_slot[u];
                    unsigned long long key = S.ckey[slot];
                    float qq = __uint_as_float((unsigned)(key >> 32));
                    if ((T)qq >= (T)stopf) break;
                    int j = (int)(key & 0xffffffffu);
                    int oid = reinterpret_cast<int *>(S.ftab)[slot];
                    int ox = (oid & 127) - 63, oy = ((oid >> 7) & 127) - 63, oz = ((oid >> 14) & 127) - 63;
                    float4 pj = __ldg(&st.p32[j]);
                    float qx, qy, qz, q2;
                    cand32(g, ci, pj, ox, oy, oz, qx, qy, qz, q2);
                    int o3[3] = {ox, oy, oz}, kk, m[3];
                    resolve(g, ci, o3, kk, m);
                    if (q2 < 1e-30f) { C.dup = true; continue; }
                    float c = 0.5f * (q2 + ci.rp32 * ci.rp32 - pj.w * pj.w);
                    int r = C.cut((T)qx, (T)qy, (T)qz, (T)c, (T)q2, j, pack_img(m[0], m[1], m[2]));
                    if (r == 2) { C.empty = true; alive = false; }
                    else if (r == 3) { C.fail = true; alive = false; }
                    else if (r == 1) stopf = (float)C.stop2();
                }
                // the ftab region is reused by the statistics below
                __syncwarp();
                if (alive && !(stopf <= rho2 * 0.9999f)) {
                    fell_back = 1;
                    alive = Driver<T, VPL, MAXP>::walk(C, g, st, off, rho2, rg, limit_hit);
                }
            } else {
                alive = Driver<T, VPL, MAXP>::walk(C, g, st, off, 0.f, rg, limit_hit);
            }
            (void)alive;
            int status = VG_CELL_OK;
            if (C.empty) status = VG_CELL_EMPTY;
            else if (C.dup) status = VG_CELL_DUP;
            else if (limit_hit) status = VG_CELL_LIMIT;
            if (!C.fail) finish<T, VPL, MAXP>(C, o, g, st, pp, status);
            if (C.degen) {
                __syncwarp();
                for (int u = lane; u < MAXP * (MAXP / 64); u += 32) (&S.u.E[0][0])[u] = 0ull;
                __syncwarp();
            }
            if (C.fail) {
                if (tier == 0 && lane == 0) {
                    int slot = atomicAdd(o.retry_count, 1);
                    o.retry[slot] = i;
                }
                if (lane == 0) {
                    int out_i = ci.self_id;
                    o.status[out_i] = VG_CELL_CAP;
                    o.nf[out_i] = 0; o.nv[out_i] = 0; o.ne[out_i] = 0;
                    o.vol[out_i] = 0; o.area[out_i] = 0;
                    o.fptr[out_i] = 0;
                }
            }
            if (pp.collect && lane == 0) {
                int out_i = ci.self_id;
                o.w_tested[out_i] = C.n_tested;
                o.w_vtests[out_i] = C.n_vtests;
                o.w_cuts[out_i] = C.n_cuts;
                o.w_retest[out_i] = C.n_retest;
                o.w_fallback[out_i] = (unsigned char)fell_back;
            }
            __syncwarp();
        }
    }
}

template <typename T, int VPL, int MAXP>
cudaError_t launch_t(const Grid &g, const Store &s, const Out &o, const Params &p, const Offsets &off,
                     unsigned *ticket, int sm_count, int warps, const int *cells, int ncells, int tier,
                     cudaStream_t st) {
    size_t smem = sizeof(Smem<T, VPL, MAXP>) * warps;
    auto kfn = k_cells3<T, VPL, MAXP>;
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, warps * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int grid = sm_count * per_sm;
    if (tier > 0) grid = sm_count;
    if ((e = cudaMemsetAsync(ticket, 0, sizeof(unsigned), st)) != cudaSuccess) return e;
    kfn<<<grid, warps * 32, smem, st>>>(g, s, o, p, off, ticket, cells, ncells, tier);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_cells3(const Grid &g, const Store &s, const Out &o, const Params &p,
                          const Offsets &off, int precision, unsigned *ticket, int sm_count,
                          int warps_per_cta, const int *cells, int ncells, int tier,
                          cudaStream_t st) {
    int w = warps_per_cta > 0 ? warps_per_cta : 4;
    if (tier > 0) return launch_t<double, 4, 128>(g, s, o, p, off, ticket, sm_count, 2, cells, ncells, tier, st);
    if (precision == VG_FP64) return launch_t<double, 2, 64>(g, s, o, p, off, ticket, sm_count, w, cells, ncells, 0, st);
    return launch_t<float, 2, 64>(g, s, o, p, off, ticket, sm_count, w, cells, ncells, 0, st);
}

}  // namespace vg
