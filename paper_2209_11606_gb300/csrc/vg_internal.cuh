// Internal declarations shared by the CUDA translation units of libvorogpu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <unordered_map>
#include <vector>

#include "vorogpu.h"

namespace vg {

constexpr unsigned FULL = 0xffffffffu;

// Blocks of up to this many particles are ordered inside by a scan over the
// block; larger ones by an in-place sort of their ids (sort_big_blocks).
constexpr int VG_SMALL_BLOCK = 64;

// Kernels launched by this host thread (every launch site increments it).
extern thread_local long long g_launch_count;

// FP64 position + radius, 32-byte aligned (one sector per particle).
struct __align__(32) D4 {
    double x, y, z, w;
};

// Geometry of a container, passed by value to kernels.
struct Grid {
    int dim;
    int per[3];       // periodic flag per axis
    int nb[3];        // blocks per axis (1 on unused axes)
    double lo[3], hi[3], L[3], h[3];
    float hf[3];      // FP32 block sides
    float Lf[3];      // FP32 box sides
    long long nblk;   // product of nb
    double s;         // mean spacing (V/N)^(1/dim)
};

// One particle system of a (possibly batched) container: its grid, where its
// blocks and particles start in the global numbering, its largest radius and
// its slice of the walk's offset list.
struct Sys {
    Grid g;
    long long blk_base;   // first global block index
    long long p_base;     // first particle, input order (systems concatenated)
    long long n;          // particles
    double rmax;          // largest radius (0 for plain Voronoi)
    int off_base, off_count, off_shell;
    int hot;              // 3D FP32 prefetch, split = 1, batched: 0 sends every
                          // cell of this system to the general kernel
};

// Sorted particle store written by the counting sort.
struct Store {
    const float4 *p32;     // block-local FP32 offset from the block's lower corner; w = radius
    const D4 *p64;         // wrapped FP64 position; w = radius
    const int *sid;        // input index of each sorted particle
    const int *sblk;       // block index of each sorted particle
    const int *bstart;     // block CSR, total blocks + 1 entries
    const int *ssys;       // system of each sorted particle
    const Sys *sys;        // system descriptors
    Sys sys0;              // system 0 by value (kernels read it from parameter space
                           // when the container has one system); its rmax is not
                           // set here: the device copy sys[0].rmax holds it
    int nsys;
    int n;                 // particles of all systems
    int radical;
};

// Per-cell outputs (indexed by input index) and the face bump buffer.
struct Out {
    double *vol, *area, *cen;     // cen: n x dim
    float *rfin;                  // R: largest vertex distance of the final cell
    int *nv, *ne, *nf;
    unsigned char *status;
    long long *fptr;              // offset of the cell's faces in `faces`
    int2 *faces;                  // {neighbour id, img bytes 0..2 | order << 24}
    unsigned long long *fcount;   // bump counter
    long long fcap;               // capacity of `faces`
    // optional work counters
    int *w_tested, *w_vtests, *w_cuts, *w_newv, *w_retest, *w_pref;
    unsigned char *w_fallback;
    int *retry;                   // sorted indices of cells for tier 1
    int *retry_count;
    int *retry2;                  // sorted indices of cells for tier 2
    int *retry2_count;
    int *retry0;                  // sorted indices of cells the hot kernel deferred (tier 3)
    int *retry0_count;
    // optional: the final cell's triangles (plane triples, 64 slots a cell)
    // and their count, 0 where the cell has merged vertices or no entry
    unsigned *topo;
    int *topo_n;
};

struct Params {
    double tol32;
    double tau_rel;
    double merge_rel;
    int prefetch_k;
    int order;
    int chunk;
    int collect;
    const float *kblock;   // per-block candidate target from the MLP, or null
    const float *rhoblk;   // per-block prefetch radius (prefetch_rho), or null
    double clip;           // clipped cells: cube side, 0 = none
    int split;             // vg_config.split (host side: which kernels run)
};

// Hardware approximations (PTX rcp/sqrt/lg2/ex2 .approx, a few ulps) where
// a value only needs a few ulps: the cell kernels' FP32 band is tol32 = 1e-5
// (about 80 ulps) wide, their statistics are checked to 1e-5, and the
// prefetch radius and its bucket bounds are heuristics or carry relative
// margins of 1e-4.
__device__ __forceinline__ float rcp_a(float x) {
    float r;
    asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float sqrt_a(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// x^(1/3) = 2^(log2(x) / 3), x > 0
__device__ __forceinline__ float cbrt_a(float x) {
    float l, r;
    asm("lg2.approx.f32 %0, %1;" : "=f"(l) : "f"(x));
    l *= (1.f / 3.f);
    asm("ex2.approx.f32 %0, %1;" : "=f"(r) : "f"(l));
    return r;
}

static __device__ __noinline__ int floordiv(int a, int b) {
    int q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) q--;
    return q;
}
// floor(a / b) for b > 0, without a division when a lies within one period
// (the general case, rare, stays out of line)
// of [0, b) (block offsets of the prefetch and of the walk's near shells)
__device__ __forceinline__ int floordiv_near(int a, int b) {
    if ((unsigned)a < (unsigned)b) return 0;
    if (a < 0 && a >= -b) return -1;
    if (a >= b && a < 2 * b) return 1;
    return floordiv(a, b);
}

// The descriptor of the current cell's system: for a single-system launch
// system 0 from parameter space (constant-bank operands), else the copy a
// warp keeps in shared memory.
template <bool BATCH>
__device__ __forceinline__ const Sys &sys_ref(const Store &st, const Sys &shared_copy) {
    if constexpr (BATCH) return shared_copy;
    else return st.sys0;
}

// Sorted offset lists for the walk, one slice per system (Sys::off_base,
// off_count): offsets (dx,dy,dz) in bytes 0..2 and the lower bound of the
// distance from any point of the home block, ascending.
struct Offsets {
    const int *code;
    const float *lb;
};

// ---- launchers (return cudaError_t) ----------------------------------------

cudaError_t sort_particles(const Sys *sys, int nsys, int dim, long long total_blk, long long n,
                           const double *pos, const double *radii, int *key, int *slot, int *count,
                           int *bstart, int *tmp_id, float4 *p32, D4 *p64, int *sid, int *sblk,
                           int *ssys, int *errflags, void *scan_tmp, cudaStream_t st);
cudaError_t system_rmax(Sys *sys, int nsys, long long n, const double *radii, cudaStream_t st);
// In-place ascending sort of the particle ids of every block holding more
// than VG_SMALL_BLOCK particles (scratch: n ints; list: nblk ints; *nlist 0
// on entry).
cudaError_t sort_big_blocks(const int *bstart, long long nblk, int *ids, int *scratch, int *list, int *nlist,
                            int grid, cudaStream_t st);
// FP32 input widened to FP64 (n values), the form every sort kernel reads.
cudaError_t widen_f32(const float *in, double *out, long long n, cudaStream_t st);
size_t scan_tmp_bytes_i32(long long n);
size_t scan_tmp_bytes_i64(long long n);
cudaError_t exclusive_scan_i32(const int *in, int *out, long long n, void *tmp, cudaStream_t st);
cudaError_t exclusive_scan_i64_from_i32(const int *in, long long *out, long long n, void *tmp,
                                        cudaStream_t st);

// Weinberg codes (Sec. 4) of the cells whose topology the cell kernel stored.
cudaError_t launch_weinberg(const unsigned *topo, const int *topo_n, long long n, int *wlen,
                            unsigned long long *whash, int *wsym, int sm_count, cudaStream_t st);
cudaError_t launch_cells3(const Store &s, const Out &o, const Params &p, const Offsets &off,
                          int precision, unsigned *ticket, int sm_count, int warps_per_cta,
                          const int *cells, int ncells, int tier, cudaStream_t st);
cudaError_t launch_cells3_hot(const Store &s, const Out &o, const Params &p, const Offsets &off, unsigned *ticket,
                              int sm_count, int warps_per_cta, const int *cells, int ncells, cudaStream_t st);
// Per-block radius of the distance-sorted preload: the ball expected to hold
// the block's candidate target (kblock, else kfixed) at the density of the 27
// blocks around it.
cudaError_t prefetch_rho(const Sys *sys, int nsys, const int *bstart, long long nblk, const float *kblock,
                         float kfixed, float *rho, cudaStream_t st);
cudaError_t launch_cells2(const Store &s, const Out &o, const Params &p, const Offsets &off,
                          int precision, unsigned *ticket, int sm_count, int warps_per_cta,
                          const int *cells, int ncells, int tier, cudaStream_t st);

// Per-block preload targets from the predictor's FP16 weights (vg_mlp.cu).
cudaError_t launch_predict(const void *weights, const Sys *sys, int nsys, const int *bstart, long long nblk,
                           float alpha, float kmin, float kmax, float *kblock, cudaStream_t st);
const void *mlp_weights(const vg_mlp *m);

// Sorted positions of the input indices cells[0..m) (via the inverse of
// sid); out-of-range indices are counted in *bad and mapped to 0.
cudaError_t map_cells(const int *sid, long long n, const int *cells, long long m, int *rank, int *out, int *bad,
                      cudaStream_t st);

cudaError_t compact_faces(long long n, const int *nf, const unsigned char *status,
                          const long long *fptr, const int2 *faces, long long fcap, long long *face_off,
                          int *nbr_id, signed char *nbr_img, unsigned char *face_order,
                          void *scan_tmp, cudaStream_t st);


}  // namespace vg

// ---- the context --------------------------------------------------------------

struct vg_ctx {
    int dim = 3;
    vg::Grid g{};             // system 0 (single-system containers)
    int grid_fixed = 0;
    double n_opt = 0;
    // systems (one for vg_create, many for vg_batch_create)
    std::vector<vg::Sys> sys;
    std::vector<int> sys_fixed;     // 1: block counts given by the caller
    std::vector<double> sys_nopt;
    vg::Sys *d_sys = nullptr;         // descriptors the kernels read (r_max filled on the device)
    vg::Sys *d_sys_init = nullptr;    // the same as laid out on the host (r_max = 0)
    long long total_blk = 0;
    int batched = 0;
    cudaStream_t stream = nullptr;
    int device = 0;
    int sm_count = 0;
    std::string err;
    std::unordered_map<void *, long long> caps;  // element capacity per device buffer

    long long n = 0;          // particles inserted (all systems)
    int radical = 0;
    int inserted = 0, computed = 0;

    // per-particle device buffers
    double *d_pos = nullptr, *d_rad = nullptr;   // staged copies of host input; FP32 input widened
    float *d_pos32 = nullptr, *d_rad32 = nullptr; // host FP32 input staged before widening
    int *d_key = nullptr, *d_slot = nullptr, *d_tmp = nullptr, *d_ssys = nullptr;
    float4 *d_p32 = nullptr;
    vg::D4 *d_p64 = nullptr;
    int *d_sid = nullptr, *d_sblk = nullptr;
    int *d_count = nullptr, *d_bstart = nullptr;
    int *d_err = nullptr;          // [0] out of box, [1] non-finite
    void *d_scan = nullptr;
    size_t scan_bytes = 0;

    // outputs
    double *d_vol = nullptr, *d_area = nullptr, *d_cen = nullptr;
    int *d_nv = nullptr, *d_ne = nullptr, *d_nf = nullptr;
    unsigned char *d_status = nullptr;
    long long *d_fptr = nullptr;
    int2 *d_faces = nullptr;
    long long fcap = 0;
    unsigned long long *d_fcount = nullptr;
    unsigned *d_ticket = nullptr;
    long long *d_face_off = nullptr;
    int *d_nbr = nullptr;
    signed char *d_img = nullptr;
    unsigned char *d_ford = nullptr;
    int *d_w_tested = nullptr, *d_w_vtests = nullptr, *d_w_cuts = nullptr, *d_w_retest = nullptr;
    int *d_w_newv = nullptr, *d_w_pref = nullptr;
    float *d_rfin = nullptr;
    // Weinberg codes: kept triangles, their counts, the codes
    unsigned *d_topo = nullptr;
    int *d_topo_n = nullptr, *d_wlen = nullptr, *d_wsym = nullptr;
    unsigned long long *d_whash = nullptr;
    int wb_valid = 0;
    // event pairs around the cell kernels (time_kernels)
    static constexpr int NEV = 256;
    cudaEvent_t ev[2 * NEV] = {};
    int nev = 0;
    unsigned char *d_w_fallback = nullptr;
    int *d_caplist = nullptr, *d_capcount = nullptr;
    int *d_caplist2 = nullptr, *d_capcount2 = nullptr;
    int *d_caplist0 = nullptr, *d_capcount0 = nullptr;   // deferred by the hot 3D kernel

    // walk offsets, one slice per distinct block shape (Sys::off_base)
    int *d_off_code = nullptr;
    float *d_off_lb = nullptr;

    long long launches = 0;   // kernels launched by this context

    // vg_compute_subset: sorted position of every input index, the mapped list
    int *d_rank = nullptr, *d_subset = nullptr, *d_subset_in = nullptr;
    int subset = 0;           // the last compute covered a subset of the cells

    // CUDA graph of one whole step (sort -> cells -> faces), vg_graph_capture()
    cudaStream_t gstream = nullptr;       // capture stream (non-blocking)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    // event nodes around the cell kernels ([0], [1]) and the sort ([2], [3])
    cudaEvent_t gev[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaGraphNode_t gev_node[4] = {nullptr, nullptr, nullptr, nullptr};
    // event pairs around the sort of timed graph replays
    cudaEvent_t sev[2 * NEV] = {};
    int nsev = 0;
    long long graph_kernels = 0;          // kernels one replay launches
    int graph_timed = 0;
    int graph_unchecked = 0;              // replayed, flags not read yet
    std::vector<int64_t> g_counts;        // capture arguments, for a re-capture
    const void *g_pos = nullptr, *g_rad = nullptr;
    int g_dtype = 0;
    vg_config g_cfg{};

    // learned preload targets, one per block (valid until the next insert)
    vg_mlp *pred = nullptr;   // predictor run after every sort (vg_set_predictor)
    float pred_alpha = 1.f, pred_kmin = 8.f, pred_kmax = 1024.f;
    float *d_kblock = nullptr;
    float *d_rho = nullptr;      // per-block prefetch radius (3D FP32 prefetch)
    long long cap_kblock = 0;
    int kblock_valid = 0;
    // training data of the predictor: k* per cell, largest k* and features per block
    int *d_kstar = nullptr, *d_kmax = nullptr;
    float *d_feat = nullptr;
    long long cap_kstar = 0, cap_kmax = 0, cap_feat = 0;
};
