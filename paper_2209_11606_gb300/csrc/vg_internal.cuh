// Internal declarations shared by the CUDA translation units of libvorogpu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <unordered_map>

#include "vorogpu.h"

namespace vg {

constexpr unsigned FULL = 0xffffffffu;

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

// Sorted particle store written by the counting sort.
struct Store {
    const float4 *p32;     // block-local FP32 offset from the block's lower corner; w = radius
    const D4 *p64;         // wrapped FP64 position; w = radius
    const int *sid;        // input index of each sorted particle
    const int *sblk;       // block index of each sorted particle
    const int *bstart;     // block CSR, nblk + 1 entries
    int n;
    int radical;
    double rmax;           // largest radius (0 for plain Voronoi)
};

// Per-cell outputs (indexed by input index) and the face bump buffer.
struct Out {
    double *vol, *area, *cen;     // cen: n x dim
    int *nv, *ne, *nf;
    unsigned char *status;
    long long *fptr;              // offset of the cell's faces in `faces`
    int2 *faces;                  // {neighbour id, img bytes 0..2 | order << 24}
    unsigned long long *fcount;   // bump counter
    long long fcap;               // capacity of `faces`
    // optional work counters
    int *w_tested, *w_vtests, *w_cuts, *w_newv, *w_retest;
    unsigned char *w_fallback;
    int *retry;                   // sorted indices of cells for tier 1
    int *retry_count;
    int *retry2;                  // sorted indices of cells for tier 2
    int *retry2_count;
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
};

// Sorted offset list for the walk: offsets (dx,dy,dz) in bytes 0..2 and the
// lower bound of the distance from any point of the home block, ascending.
struct Offsets {
    const int *code;
    const float *lb;
    int count;
    int shell;   // Chebyshev radius covered by the list
};

// ---- launchers (return cudaError_t) ----------------------------------------

cudaError_t sort_particles(const Grid &g, long long n, const double *pos, const double *radii,
                           int *key, int *slot, int *count, int *bstart, int *tmp_id,
                           float4 *p32, D4 *p64, int *sid, int *sblk, int *errflags,
                           void *scan_tmp, size_t scan_tmp_bytes, cudaStream_t st);
size_t scan_tmp_bytes_i32(long long n);
size_t scan_tmp_bytes_i64(long long n);
cudaError_t exclusive_scan_i32(const int *in, int *out, long long n, void *tmp, cudaStream_t st);
cudaError_t exclusive_scan_i64_from_i32(const int *in, long long *out, long long n, void *tmp,
                                        cudaStream_t st);

cudaError_t launch_cells3(const Grid &g, const Store &s, const Out &o, const Params &p,
                          const Offsets &off, int precision, unsigned *ticket, int sm_count,
                          int warps_per_cta, const int *cells, int ncells, int tier,
                          cudaStream_t st);
cudaError_t launch_cells2(const Grid &g, const Store &s, const Out &o, const Params &p,
                          const Offsets &off, int precision, unsigned *ticket, int sm_count,
                          int warps_per_cta, const int *cells, int ncells, int tier,
                          cudaStream_t st);

cudaError_t compact_faces(long long n, const int *nf, const unsigned char *status,
                          const long long *fptr, const int2 *faces, long long *face_off,
                          int *nbr_id, signed char *nbr_img, unsigned char *face_order,
                          void *scan_tmp, cudaStream_t st);


}  // namespace vg

// ---- the context --------------------------------------------------------------

struct vg_ctx {
    int dim = 3;
    vg::Grid g{};
    int grid_fixed = 0;
    double n_opt = 0;
    cudaStream_t stream = nullptr;
    int device = 0;
    int sm_count = 0;
    std::string err;
    std::unordered_map<void *, long long> caps;  // element capacity per device buffer

    long long n = 0;          // particles inserted
    long long cap_n = 0;      // capacity of per-particle buffers
    long long cap_blk = 0;
    int radical = 0;
    double rmax = 0;
    int inserted = 0, computed = 0;

    // per-particle device buffers
    double *d_pos = nullptr, *d_rad = nullptr;   // staged copies of host input
    int *d_key = nullptr, *d_slot = nullptr, *d_tmp = nullptr;
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
    long long cap_faces_csr = 0;
    int *d_w_tested = nullptr, *d_w_vtests = nullptr, *d_w_cuts = nullptr, *d_w_retest = nullptr;
    int *d_w_newv = nullptr;
    // event pairs around the cell kernels (time_kernels)
    static constexpr int NEV = 256;
    cudaEvent_t ev[2 * NEV] = {};
    int nev = 0;
    unsigned char *d_w_fallback = nullptr;
    int *d_caplist = nullptr, *d_capcount = nullptr;
    int *d_caplist2 = nullptr, *d_capcount2 = nullptr;
    long long total_faces = -1;

    // walk offsets
    int *d_off_code = nullptr;
    float *d_off_lb = nullptr;
    int off_count = 0, off_shell = 0;

    long long launches = 0;   // kernels launched by this context

    // MLP per-block predictions
    float *d_kblock = nullptr;
    long long cap_kblock = 0;
};
