// Host side of the C ABI declared in include/vorogpu.h: argument checks,
// device buffers, the sort -> cells -> faces pipeline, and result copies.
//
// A container holds one or more independent particle systems (vg_create: one;
// vg_batch_create: many).  Their blocks and particles are numbered globally,
// system after system, so one counting sort and one persistent cell launch
// (cells taken from one atomic work queue) serve all of them.
#include <math.h>
#include <stddef.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "vg_internal.cuh"

using namespace vg;

namespace vg {
thread_local long long g_launch_count = 0;
}

namespace {

vg_status fail(vg_ctx *c, vg_status s, const std::string &msg) {
    if (c) c->err = msg;
    return s;
}

vg_status cuda_fail(vg_ctx *c, cudaError_t e, const char *where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(c, e == cudaErrorMemoryAllocation ? VG_ERR_OOM : VG_ERR_CUDA, m);
}

#define VG_CUDA(call)                                          \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #call); \
    } while (0)

// Grows a context-owned device buffer to hold `need` elements; each buffer
// keeps its own capacity, so repeated inserts of one size never reallocate.
template <typename T>
cudaError_t ensure(vg_ctx *c, T *&p, long long need) {
    long long &cap = c->caps[(void *)&p];
    if (p && need <= cap) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    long long n = std::max<long long>(need, 1);
    cudaError_t e = cudaMalloc((void **)&p, sizeof(T) * (size_t)n);
    if (e == cudaSuccess) cap = n;
    return e;
}

template <typename T>
void release(T *&p) {
    if (p) cudaFree(p);
    p = nullptr;
}

// Block counts from n_opt (Sec. 2.1.4), floor rounding as in Table 3.
void grid_from_nopt(Grid &g, int dim, double n_opt, long long n) {
    double V = 1;
    for (int a = 0; a < dim; a++) V *= g.L[a];
    const double nopt = n_opt > 0 ? n_opt : (dim == 3 ? 4.6 : 3.4);
    const double lam = pow((double)std::max<long long>(n, 1) / (nopt * V), 1.0 / dim);
    for (int a = 0; a < dim; a++) {
        const long long v = (long long)floor(lam * g.L[a]);
        g.nb[a] = (int)std::max<long long>(1, std::min<long long>(v, 1 << 20));
    }
}

void finish_grid(Grid &g, int dim) {
    g.dim = dim;
    g.nblk = 1;
    for (int a = 0; a < 3; a++) {
        if (a >= dim) { g.nb[a] = 1; g.lo[a] = 0; g.hi[a] = 1; g.L[a] = 1; g.per[a] = 0; }
        g.h[a] = g.L[a] / g.nb[a];
        g.hf[a] = (float)g.h[a];
        g.Lf[a] = (float)g.L[a];
        g.nblk *= g.nb[a];
    }
}

// Appends the sorted list of block offsets for the walk of one grid: all
// offsets whose distance bound from the home block lies below shell * h_min,
// ascending by that bound (then by L1 length).
void offsets_for(const Grid &g, int dim, int S, std::vector<int> &code, std::vector<float> &lbv) {
    double hmin = 1e300;
    for (int a = 0; a < dim; a++) hmin = std::min(hmin, g.h[a]);
    struct E { float lb; int l1; int code; };
    std::vector<E> v;
    int lim[3];
    for (int a = 0; a < 3; a++) lim[a] = a < dim ? S : 0;
    for (int z = -lim[2]; z <= lim[2]; z++)
        for (int y = -lim[1]; y <= lim[1]; y++)
            for (int x = -lim[0]; x <= lim[0]; x++) {
                const int o[3] = {x, y, z};
                double lb2 = 0;
                for (int a = 0; a < 3; a++) {
                    const double t = std::max(0, std::abs(o[a]) - 1) * (double)g.hf[a];
                    lb2 += t * t;
                }
                // the kernels' shell continuation skips offsets whose FP32
                // bound is below shell*h_min; keep exactly those here
                const float lbx = fmaxf(0.f, (float)(std::abs(x) - 1)) * g.hf[0];
                const float lby = fmaxf(0.f, (float)(std::abs(y) - 1)) * g.hf[1];
                const float lbz = fmaxf(0.f, (float)(std::abs(z) - 1)) * g.hf[2];
                const float lbmax = (float)S * (float)hmin;
                if (!(lbx * lbx + lby * lby + lbz * lbz < lbmax * lbmax)) continue;
                v.push_back({(float)sqrt(lb2), std::abs(x) + std::abs(y) + std::abs(z),
                             (x & 0xff) | ((y & 0xff) << 8) | ((z & 0xff) << 16)});
            }
    std::stable_sort(v.begin(), v.end(), [](const E &a, const E &b) {
        if (a.lb != b.lb) return a.lb < b.lb;
        return a.l1 < b.l1;
    });
    for (const E &e : v) { code.push_back(e.code); lbv.push_back(e.lb); }
}

bool same_offsets(const Grid &a, const Grid &b, int dim) {
    for (int k = 0; k < dim; k++)
        if (a.hf[k] != b.hf[k] || a.h[k] != b.h[k]) return false;
    return true;
}

// Fixes every system's grid (the n_opt rule where not given), numbers the
// blocks and particles globally, builds the offset lists and uploads the
// descriptors.  r_max starts at 0; system_rmax() fills it on the device.
vg_status layout_systems(vg_ctx *c, const std::vector<long long> &counts) {
    const int d = c->dim;
    std::vector<int> code;
    std::vector<float> lbv;
    long long blk = 0, pbase = 0;
    const int S = 4;
    for (size_t k = 0; k < c->sys.size(); k++) {
        Sys &s = c->sys[k];
        if (!c->sys_fixed[k]) grid_from_nopt(s.g, d, c->sys_nopt[k], counts[k]);
        finish_grid(s.g, d);
        double V = 1;
        for (int a = 0; a < d; a++) V *= s.g.L[a];
        s.g.s = pow(V / (double)std::max<long long>(counts[k], 1), 1.0 / d);
        s.blk_base = blk;
        s.p_base = pbase;
        s.n = counts[k];
        s.rmax = 0;
        blk += s.g.nblk;
        pbase += counts[k];
        // systems with the same block sides share one offset list
        int shared = -1;
        for (size_t q = 0; q < k && shared < 0; q++)
            if (same_offsets(c->sys[q].g, s.g, d)) shared = (int)q;
        if (shared >= 0) {
            s.off_base = c->sys[shared].off_base;
            s.off_count = c->sys[shared].off_count;
        } else {
            s.off_base = (int)code.size();
            offsets_for(s.g, d, S, code, lbv);
            s.off_count = (int)code.size() - s.off_base;
        }
        s.off_shell = S;
    }
    if (blk > (1ll << 31) - 2) return fail(c, VG_ERR_ARG, "too many blocks in total");
    c->total_blk = blk;
    c->g = c->sys[0].g;
    VG_CUDA(ensure(c, c->d_off_code, (long long)code.size()));
    VG_CUDA(ensure(c, c->d_off_lb, (long long)lbv.size()));
    VG_CUDA(ensure(c, c->d_sys, (long long)c->sys.size()));
    VG_CUDA(ensure(c, c->d_sys_init, (long long)c->sys.size()));
    VG_CUDA(cudaMemcpyAsync(c->d_off_code, code.data(), sizeof(int) * code.size(), cudaMemcpyHostToDevice,
                            c->stream));
    VG_CUDA(cudaMemcpyAsync(c->d_off_lb, lbv.data(), sizeof(float) * lbv.size(), cudaMemcpyHostToDevice, c->stream));
    VG_CUDA(cudaMemcpyAsync(c->d_sys_init, c->sys.data(), sizeof(Sys) * c->sys.size(), cudaMemcpyHostToDevice,
                            c->stream));
    // the host vectors must outlive the asynchronous copies
    VG_CUDA(cudaStreamSynchronize(c->stream));
    return VG_OK;
}

vg_status copy_out(vg_ctx *c, void *dst, const void *src, size_t bytes, int on_device) {
    if (!dst || bytes == 0) return VG_OK;
    if (on_device) {
        VG_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, c->stream));
    } else {
        VG_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c->stream));
        VG_CUDA(cudaStreamSynchronize(c->stream));
    }
    return VG_OK;
}

bool box_ok(int dim, const double *lo, const double *hi) {
    for (int a = 0; a < dim; a++)
        if (!isfinite(lo[a]) || !isfinite(hi[a]) || !(hi[a] > lo[a])) return false;
    return true;
}

// A context on the current device with its small fixed buffers.
vg_status new_context(vg_ctx **made, int dim, void *stream) {
    *made = nullptr;
    vg_ctx *c = new (std::nothrow) vg_ctx();
    if (!c) return VG_ERR_OOM;
    c->dim = dim;
    c->stream = (cudaStream_t)stream;
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return VG_ERR_CUDA;
    }
    cudaError_t e = cudaMalloc((void **)&c->d_err, sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_fcount, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_ticket, sizeof(unsigned) * 4);
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_capcount, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_capcount2, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_capcount0, sizeof(int));
    if (e != cudaSuccess) {
        cudaGetLastError();
        vg_destroy(c);
        return e == cudaErrorMemoryAllocation ? VG_ERR_OOM : VG_ERR_CUDA;
    }
    *made = c;
    return VG_OK;
}

void release_graph(vg_ctx *c) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->gexec = nullptr;
    c->graph = nullptr;
    for (int k = 0; k < 4; k++) c->gev_node[k] = nullptr;
    c->graph_unchecked = 0;
}

// Host half of an insert: validation, layout of the systems, buffers, and
// the copy of host input to the device.  Returns the device input pointers
// (of type `dtype`; FP32 input is widened by enqueue_sort).
vg_status prepare_insert(vg_ctx *c, const std::vector<long long> &counts, const void *pos, const void *radii,
                         int dtype, int on_device, const void **dpos, const void **drad) {
    long long n = 0;
    for (long long k : counts) n += k;
    if (n > 0x7ffffffe) return fail(c, VG_ERR_ARG, "particle count out of range");
    if (n > 0 && !pos) return fail(c, VG_ERR_ARG, "pos is NULL");
    if (dtype != VG_F64 && dtype != VG_F32) return fail(c, VG_ERR_ARG, "dtype must be VG_F64 or VG_F32");
    // buffers may move below: a captured graph would point at freed memory
    release_graph(c);
    c->inserted = 0;
    c->kblock_valid = 0;
    c->subset = 0;
    c->computed = 0;
    c->wb_valid = 0;
    const int d = c->dim;
    vg_status ls = layout_systems(c, counts);
    if (ls != VG_OK) return ls;
    VG_CUDA(ensure(c, c->d_key, n));
    VG_CUDA(ensure(c, c->d_slot, n));
    VG_CUDA(ensure(c, c->d_tmp, n));
    VG_CUDA(ensure(c, c->d_p32, n));
    VG_CUDA(ensure(c, c->d_p64, n));
    VG_CUDA(ensure(c, c->d_sid, n));
    VG_CUDA(ensure(c, c->d_sblk, n));
    VG_CUDA(ensure(c, c->d_ssys, n));
    VG_CUDA(ensure(c, c->d_vol, n));
    VG_CUDA(ensure(c, c->d_area, n));
    VG_CUDA(ensure(c, c->d_cen, n * 3));
    VG_CUDA(ensure(c, c->d_nv, n));
    VG_CUDA(ensure(c, c->d_ne, n));
    VG_CUDA(ensure(c, c->d_nf, n));
    VG_CUDA(ensure(c, c->d_status, n));
    VG_CUDA(ensure(c, c->d_fptr, n));
    VG_CUDA(ensure(c, c->d_face_off, n + 1));
    VG_CUDA(ensure(c, c->d_caplist, n));
    VG_CUDA(ensure(c, c->d_caplist2, n));
    VG_CUDA(ensure(c, c->d_caplist0, n));
    VG_CUDA(ensure(c, c->d_w_tested, n));
    VG_CUDA(ensure(c, c->d_w_vtests, n));
    VG_CUDA(ensure(c, c->d_w_cuts, n));
    VG_CUDA(ensure(c, c->d_w_retest, n));
    VG_CUDA(ensure(c, c->d_w_newv, n));
    VG_CUDA(ensure(c, c->d_w_pref, n));
    VG_CUDA(ensure(c, c->d_rfin, n));
    VG_CUDA(ensure(c, c->d_w_fallback, n));
    // FP64 staging: host FP64 input is copied there, FP32 input (host or
    // device) is widened into it
    if (!on_device || dtype == VG_F32) {
        VG_CUDA(ensure(c, c->d_pos, n * d));
        if (radii) VG_CUDA(ensure(c, c->d_rad, n));
    }
    if (!on_device && dtype == VG_F32) {
        VG_CUDA(ensure(c, c->d_pos32, n * d));
        if (radii) VG_CUDA(ensure(c, c->d_rad32, n));
    }
    VG_CUDA(ensure(c, c->d_count, c->total_blk));
    if (c->pred) {
        if (!c->d_kblock || c->cap_kblock < c->total_blk) {
            if (c->d_kblock) cudaFree(c->d_kblock);
            c->d_kblock = nullptr;
            c->cap_kblock = 0;
            VG_CUDA(cudaMalloc((void **)&c->d_kblock, sizeof(float) * std::max<long long>(1, c->total_blk)));
            c->cap_kblock = c->total_blk;
        }
    }
    VG_CUDA(ensure(c, c->d_bstart, c->total_blk + 1));
    VG_CUDA(ensure(c, c->d_rho, c->total_blk));
    const size_t need_scan = std::max(scan_tmp_bytes_i32(c->total_blk + 1),
                                      (((size_t)n * sizeof(int) + 255) & ~(size_t)255) + scan_tmp_bytes_i64(n + 1));
    if (need_scan > c->scan_bytes) {
        if (c->d_scan) cudaFree(c->d_scan);
        c->d_scan = nullptr;
        c->scan_bytes = 0;
        VG_CUDA(cudaMalloc(&c->d_scan, need_scan));
        c->scan_bytes = need_scan;
    }
    *dpos = pos;
    *drad = radii;
    if (n > 0 && !on_device) {
        const size_t es = dtype == VG_F32 ? sizeof(float) : sizeof(double);
        void *stage_p = dtype == VG_F32 ? (void *)c->d_pos32 : (void *)c->d_pos;
        void *stage_r = dtype == VG_F32 ? (void *)c->d_rad32 : (void *)c->d_rad;
        VG_CUDA(cudaMemcpyAsync(stage_p, pos, es * n * d, cudaMemcpyHostToDevice, c->stream));
        *dpos = stage_p;
        if (radii) {
            VG_CUDA(cudaMemcpyAsync(stage_r, radii, es * n, cudaMemcpyHostToDevice, c->stream));
            *drad = stage_r;
        }
    }
    c->n = n;
    c->radical = radii != nullptr;
    return VG_OK;
}

// Device half of an insert: FP32 input widened to FP64, then the counting
// sort of all systems, enqueued on `s` with no host synchronisation (so it
// can be captured in a graph).
cudaError_t enqueue_sort(vg_ctx *c, const void *src_pos, const void *src_rad, int dtype, cudaStream_t s) {
    const int nsys = (int)c->sys.size();
    const double *dpos = (const double *)src_pos, *drad = (const double *)src_rad;
    cudaError_t e = cudaSuccess;
    if (dtype == VG_F32) {
        e = widen_f32((const float *)src_pos, c->d_pos, c->n * c->dim, s);
        dpos = c->d_pos;
        if (e == cudaSuccess && src_rad) {
            e = widen_f32((const float *)src_rad, c->d_rad, c->n, s);
            drad = c->d_rad;
        }
        if (e != cudaSuccess) return e;
    }
    // fresh descriptors: r_max is accumulated from 0 by system_rmax
    e = cudaMemcpyAsync(c->d_sys, c->d_sys_init, sizeof(Sys) * nsys, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && drad) e = system_rmax(c->d_sys, nsys, c->n, drad, s);
    if (e == cudaSuccess)
        e = sort_particles(c->d_sys, nsys, c->dim, c->total_blk, c->n, dpos, drad, c->d_key, c->d_slot, c->d_count,
                           c->d_bstart, c->d_tmp, c->d_p32, c->d_p64, c->d_sid, c->d_sblk, c->d_ssys, c->d_err,
                           c->d_scan, s);
    // the learned preload targets follow the block counts
    if (e == cudaSuccess && c->pred)
        e = launch_predict(mlp_weights(c->pred), c->d_sys, nsys, c->d_bstart, c->total_blk, c->pred_alpha,
                           c->pred_kmin, c->pred_kmax, c->d_kblock, s);
    return e;
}

// Input errors the sort flagged (read after the stream has drained).
vg_status read_input_flags(vg_ctx *c) {
    int herr[2] = {0, 0};
    VG_CUDA(cudaMemcpyAsync(herr, c->d_err, sizeof(int) * 2, cudaMemcpyDeviceToHost, c->stream));
    VG_CUDA(cudaStreamSynchronize(c->stream));
    if (herr[1]) return fail(c, VG_ERR_NONFINITE, std::to_string(herr[1]) + " non-finite coordinates or radii");
    if (herr[0]) return fail(c, VG_ERR_OUT_OF_BOX, std::to_string(herr[0]) + " particles outside a walled box");
    return VG_OK;
}

// Shared by vg_insert and vg_batch_insert: counts[k] particles of system k,
// all systems' rows concatenated in `pos` / `radii`.
vg_status insert_all(vg_ctx *c, const std::vector<long long> &counts, const void *pos, const void *radii,
                     int dtype, int on_device) {
    const void *dpos = nullptr, *drad = nullptr;
    vg_status s = prepare_insert(c, counts, pos, radii, dtype, on_device, &dpos, &drad);
    if (s != VG_OK) return s;
    const long long l0 = g_launch_count;
    cudaError_t e = enqueue_sort(c, dpos, drad, dtype, c->stream);
    c->launches += g_launch_count - l0;
    if (e != cudaSuccess) return cuda_fail(c, e, "sort_particles");
    if ((s = read_input_flags(c)) != VG_OK) return s;
    c->inserted = 1;
    if (c->pred) c->kblock_valid = 1;
    return VG_OK;
}

// `inserts`: the call inserts first (a graph capture), so an attached
// predictor supplies the per-block preload targets itself.
vg_status check_config(vg_ctx *c, const vg_config &cfg, bool inserts = false) {
    if (cfg.precision != VG_FP64 && cfg.precision != VG_FP32_RETEST) return fail(c, VG_ERR_ARG, "precision");
    if (cfg.order != VG_WALK && cfg.order != VG_PREFETCH) return fail(c, VG_ERR_ARG, "order");
    if (!(cfg.tol32 > 0) || !(cfg.tau_rel > 0) || !(cfg.merge_rel > 0)) return fail(c, VG_ERR_ARG, "tolerances");
    if (!(cfg.clip >= 0) || !(cfg.clip < 1e300)) return fail(c, VG_ERR_ARG, "clip must be finite and >= 0");
    if (cfg.weinberg && c->dim != 3) return fail(c, VG_ERR_ARG, "Weinberg codes: 3D cells");
    if (cfg.warps_per_cta > 4) return fail(c, VG_ERR_ARG, "warps_per_cta above 4 (CTAs of at most 128 threads)");
    if (cfg.use_mlp && !c->kblock_valid && !(inserts && c->pred))
        return fail(c, VG_ERR_STATE, "use_mlp without vg_mlp_predict after the insert");
    return VG_OK;
}

// The three cell launches (tier 0 over all cells, then the large-cell
// tiers over the cells the previous tier handed on), enqueued on `s`.
cudaError_t enqueue_cells(vg_ctx *c, const vg_config &cfg, cudaStream_t s, const int *subset = nullptr,
                          int nsubset = 0) {
    Store st;
    st.p32 = c->d_p32; st.p64 = c->d_p64; st.sid = c->d_sid; st.sblk = c->d_sblk; st.bstart = c->d_bstart;
    st.ssys = c->d_ssys; st.sys = c->d_sys; st.sys0 = c->sys[0]; st.nsys = (int)c->sys.size();
    st.n = (int)c->n; st.radical = c->radical;
    Params pp;
    pp.tol32 = cfg.tol32; pp.tau_rel = cfg.tau_rel; pp.merge_rel = cfg.merge_rel;
    pp.clip = cfg.clip;
    pp.prefetch_k = cfg.prefetch_k; pp.order = cfg.order;
    pp.chunk = cfg.chunk > 0 ? cfg.chunk : 1;
    pp.collect = cfg.collect_stats ? 1 : 0;
    pp.kblock = cfg.use_mlp ? c->d_kblock : nullptr;
    pp.rhoblk = c->d_rho;
    pp.split = cfg.split ? 1 : 0;
    Offsets off;
    off.code = c->d_off_code; off.lb = c->d_off_lb;
    Out o;
    o.vol = c->d_vol; o.area = c->d_area; o.cen = c->d_cen; o.rfin = c->d_rfin;
    o.nv = c->d_nv; o.ne = c->d_ne; o.nf = c->d_nf; o.status = c->d_status;
    o.fptr = c->d_fptr; o.faces = c->d_faces; o.fcount = c->d_fcount; o.fcap = c->fcap;
    o.w_tested = c->d_w_tested; o.w_vtests = c->d_w_vtests; o.w_cuts = c->d_w_cuts;
    o.w_retest = c->d_w_retest; o.w_fallback = c->d_w_fallback; o.w_newv = c->d_w_newv;
    o.w_pref = c->d_w_pref;
    o.retry = c->d_caplist; o.retry_count = c->d_capcount;
    o.retry2 = c->d_caplist2; o.retry2_count = c->d_capcount2;
    o.retry0 = c->d_caplist0; o.retry0_count = c->d_capcount0;
    o.topo = cfg.weinberg ? c->d_topo : nullptr;
    o.topo_n = cfg.weinberg ? c->d_topo_n : nullptr;
    cudaError_t e;
    if (cfg.weinberg && (e = cudaMemsetAsync(c->d_topo_n, 0, sizeof(int) * c->n, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c->d_fcount, 0, sizeof(unsigned long long), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c->d_capcount, 0, sizeof(int), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c->d_capcount2, 0, sizeof(int), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c->d_capcount0, 0, sizeof(int), s)) != cudaSuccess) return e;
    // 3D FP32 prefetch: every block's preload radius first
    if (c->dim == 3 && cfg.precision == VG_FP32_RETEST && cfg.order == VG_PREFETCH &&
        (e = prefetch_rho(c->d_sys, (int)c->sys.size(), c->d_bstart, c->total_blk, pp.kblock,
                          (float)(cfg.prefetch_k > 0 ? cfg.prefetch_k : 72), c->d_rho, s)) != cudaSuccess)
        return e;
    auto launch = c->dim == 3 ? launch_cells3 : launch_cells2;
    const int nc = subset ? nsubset : (int)c->n;
    // 3D FP32 prefetch: the hot kernel over every cell, then the general one
    // over the cells it deferred (walk after the preload, FP64 statistics)
    const bool hot = cfg.split && c->dim == 3 && cfg.precision == VG_FP32_RETEST && cfg.order == VG_PREFETCH &&
                     (!cfg.weinberg || c->sys.size() == 1) && c->n < (1 << 27);
    if (hot) {
        if ((e = launch_cells3_hot(st, o, pp, off, c->d_ticket, c->sm_count, cfg.warps_per_cta, subset, nc, s)))
            return e;
        if ((e = launch(st, o, pp, off, cfg.precision, c->d_ticket + 3, c->sm_count, cfg.warps_per_cta, c->d_caplist0,
                        0, 3, s)))
            return e;
    } else if ((e = launch(st, o, pp, off, cfg.precision, c->d_ticket, c->sm_count, cfg.warps_per_cta, subset, nc, 0,
                           s))) {
        return e;
    }
    if ((e = launch(st, o, pp, off, cfg.precision, c->d_ticket + 1, c->sm_count, 0, c->d_caplist, 0, 1, s))) return e;
    return launch(st, o, pp, off, cfg.precision, c->d_ticket + 2, c->sm_count, 0, c->d_caplist2, 0, 2, s);
}

// CSR of the faces the cell kernels wrote.
cudaError_t enqueue_compact(vg_ctx *c, cudaStream_t s) {
    return compact_faces(c->n, c->d_nf, c->d_status, c->d_fptr, c->d_faces, c->fcap, c->d_face_off, c->d_nbr,
                         c->d_img, c->d_ford, c->d_scan, s);
}

vg_status ensure_csr(vg_ctx *c) {
    VG_CUDA(ensure(c, c->d_nbr, c->fcap));
    VG_CUDA(ensure(c, c->d_img, 3 * c->fcap));
    VG_CUDA(ensure(c, c->d_ford, c->fcap));
    return VG_OK;
}

vg_status graph_check(vg_ctx *c);

}  // namespace

extern "C" {

void vg_config_default(vg_config *cfg) {
    if (!cfg) return;
    memset(cfg, 0, sizeof *cfg);
    cfg->precision = VG_FP32_RETEST;
    cfg->order = VG_PREFETCH;
    cfg->tol32 = 1e-5;
    cfg->tau_rel = 1e-11;
    cfg->merge_rel = 1e-9;
    cfg->clip = 0.0;
    cfg->weinberg = 0;
    cfg->prefetch_k = 0;
    cfg->use_mlp = 0;
    cfg->chunk = 0;
    cfg->warps_per_cta = 0;
    cfg->collect_stats = 0;
    cfg->time_kernels = 0;
    cfg->split = 1;
}

vg_status vg_create(vg_ctx **out, int dim, const double *lo, const double *hi, const int *periodic,
                    const int *nblocks, double n_opt, void *stream) {
    if (!out) return VG_ERR_ARG;
    *out = nullptr;
    if (dim != 2 && dim != 3) return VG_ERR_ARG;
    if (!lo || !hi || !periodic || !box_ok(dim, lo, hi)) return VG_ERR_ARG;
    if (nblocks) {
        long long prod = 1;
        for (int a = 0; a < dim; a++) {
            if (nblocks[a] < 1 || nblocks[a] > (1 << 20)) return VG_ERR_ARG;
            prod *= nblocks[a];
        }
        if (prod > (1ll << 30)) return VG_ERR_ARG;
    }
    vg_ctx *c = nullptr;
    vg_status s = new_context(&c, dim, stream);
    if (s != VG_OK) return s;
    Sys sy{};
    sy.hot = 1;
    for (int a = 0; a < dim; a++) {
        sy.g.lo[a] = lo[a];
        sy.g.hi[a] = hi[a];
        sy.g.L[a] = hi[a] - lo[a];
        sy.g.per[a] = periodic[a] ? 1 : 0;
        sy.g.nb[a] = nblocks ? nblocks[a] : 1;
    }
    finish_grid(sy.g, dim);
    c->sys.push_back(sy);
    c->sys_fixed.push_back(nblocks ? 1 : 0);
    c->sys_nopt.push_back(n_opt);
    c->grid_fixed = nblocks ? 1 : 0;
    c->n_opt = n_opt;
    c->g = sy.g;
    *out = c;
    return VG_OK;
}

vg_status vg_batch_create(vg_ctx **out, int dim, int nsys, const vg_system *systems, void *stream) {
    if (!out) return VG_ERR_ARG;
    *out = nullptr;
    if ((dim != 2 && dim != 3) || nsys < 1 || !systems) return VG_ERR_ARG;
    std::vector<int> fixed(nsys, 1);
    for (int k = 0; k < nsys; k++) {
        if (!box_ok(dim, systems[k].lo, systems[k].hi)) return VG_ERR_ARG;
        long long prod = 1;
        for (int a = 0; a < dim; a++) {
            if (systems[k].nblocks[a] <= 0) fixed[k] = 0;
            if (systems[k].nblocks[a] > (1 << 20)) return VG_ERR_ARG;
            prod *= std::max(1, systems[k].nblocks[a]);
        }
        if (prod > (1ll << 30)) return VG_ERR_ARG;
    }
    vg_ctx *c = nullptr;
    vg_status s = new_context(&c, dim, stream);
    if (s != VG_OK) return s;
    c->batched = 1;
    c->sys.reserve(nsys);
    for (int k = 0; k < nsys; k++) {
        const vg_system &in = systems[k];
        Sys sy{};
        sy.hot = 1;
        for (int a = 0; a < dim; a++) {
            sy.g.lo[a] = in.lo[a];
            sy.g.hi[a] = in.hi[a];
            sy.g.L[a] = in.hi[a] - in.lo[a];
            sy.g.per[a] = in.periodic[a] ? 1 : 0;
            sy.g.nb[a] = fixed[k] ? in.nblocks[a] : 1;
        }
        finish_grid(sy.g, dim);
        c->sys.push_back(sy);
        c->sys_fixed.push_back(fixed[k]);
        c->sys_nopt.push_back(in.n_opt);
    }
    c->g = c->sys[0].g;
    *out = c;
    return VG_OK;
}

vg_status vg_insert(vg_ctx *c, int64_t n, const void *pos, const void *radii, int dtype, int on_device) {
    if (!c) return VG_ERR_ARG;
    if (c->batched) return fail(c, VG_ERR_STATE, "batched container: use vg_batch_insert");
    if (n < 0) return fail(c, VG_ERR_ARG, "negative particle count");
    std::vector<long long> counts(1, (long long)n);
    return insert_all(c, counts, pos, radii, dtype, on_device);
}

vg_status vg_batch_insert(vg_ctx *c, const int64_t *counts, const void *pos, const void *radii, int dtype,
                          int on_device) {
    if (!c) return VG_ERR_ARG;
    if (!counts) return fail(c, VG_ERR_ARG, "counts is NULL");
    std::vector<long long> cv(c->sys.size());
    for (size_t k = 0; k < cv.size(); k++) {
        if (counts[k] < 0) return fail(c, VG_ERR_ARG, "negative particle count");
        cv[k] = counts[k];
    }
    return insert_all(c, cv, pos, radii, dtype, on_device);
}

vg_status vg_compute(vg_ctx *c, const vg_config *cfg_in) {
    if (!c) return VG_ERR_ARG;
    if (!c->inserted) return fail(c, VG_ERR_STATE, "vg_compute before vg_insert");
    vg_config cfg;
    if (cfg_in) cfg = *cfg_in; else vg_config_default(&cfg);
    vg_status s = check_config(c, cfg);
    if (s != VG_OK) return s;
    if (c->graph_unchecked && (s = graph_check(c)) != VG_OK) return s;
    // the face buffer may grow below: drop a captured graph
    release_graph(c);
    const long long n = c->n;
    const long long l0 = g_launch_count;
    c->wb_valid = 0;
    if (cfg.weinberg) {
        VG_CUDA(ensure(c, c->d_topo, n * 64));
        VG_CUDA(ensure(c, c->d_topo_n, n));
        VG_CUDA(ensure(c, c->d_wlen, n));
        VG_CUDA(ensure(c, c->d_wsym, n));
        VG_CUDA(ensure(c, c->d_whash, n));
    }
    // face buffer: start at 24 faces per cell, grow on overflow
    const long long want = std::max<long long>(1024, n * 24);
    if (c->fcap < want) {
        VG_CUDA(ensure(c, c->d_faces, want));
        c->fcap = want;
    }
    for (int attempt = 0; attempt < 4; attempt++) {
        const bool timed = cfg.time_kernels && c->nev < vg_ctx::NEV;
        if (timed) {
            for (int k = 0; k < 2; k++)
                if (!c->ev[2 * c->nev + k]) VG_CUDA(cudaEventCreate(&c->ev[2 * c->nev + k]));
            VG_CUDA(cudaEventRecord(c->ev[2 * c->nev], c->stream));
        }
        cudaError_t e = enqueue_cells(c, cfg, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "cell kernels");
        if (timed) {
            VG_CUDA(cudaEventRecord(c->ev[2 * c->nev + 1], c->stream));
            c->nev++;
        }
        unsigned long long used = 0;
        VG_CUDA(cudaMemcpyAsync(&used, c->d_fcount, sizeof used, cudaMemcpyDeviceToHost, c->stream));
        VG_CUDA(cudaStreamSynchronize(c->stream));
        if ((long long)used <= c->fcap) break;
        if (attempt == 3) return fail(c, VG_ERR_CAP, "face buffer overflow");
        // face buffer too small: grow to what was asked for and recompute
        const long long need = (long long)(used * 5 / 4) + 1024;
        VG_CUDA(ensure(c, c->d_faces, need));
        c->fcap = need;
    }
    if ((s = ensure_csr(c)) != VG_OK) return s;
    if (cfg.weinberg) {
        cudaError_t ew = launch_weinberg(c->d_topo, c->d_topo_n, n, c->d_wlen, c->d_whash, c->d_wsym, c->sm_count,
                                         c->stream);
        if (ew != cudaSuccess) return cuda_fail(c, ew, "weinberg");
        c->wb_valid = 1;
    }
    cudaError_t e = enqueue_compact(c, c->stream);
    c->launches += g_launch_count - l0;
    if (e != cudaSuccess) return cuda_fail(c, e, "compact_faces");
    c->computed = 1;
    c->subset = 0;
    return VG_OK;
}

vg_status vg_compute_subset(vg_ctx *c, const vg_config *cfg_in, const int32_t *cells, int64_t m, int on_device) {
    if (!c) return VG_ERR_ARG;
    if (!c->inserted) return fail(c, VG_ERR_STATE, "vg_compute_subset before vg_insert");
    vg_config cfg;
    if (cfg_in) cfg = *cfg_in; else vg_config_default(&cfg);
    vg_status s = check_config(c, cfg);
    if (s != VG_OK) return s;
    if (cfg.weinberg) return fail(c, VG_ERR_ARG, "Weinberg codes: vg_compute only");
    if (m < 0 || m > c->n || (m > 0 && !cells)) return fail(c, VG_ERR_ARG, "bad cell list");
    if (c->graph_unchecked && (s = graph_check(c)) != VG_OK) return s;
    release_graph(c);
    const long long n = c->n;
    const long long l0 = g_launch_count;
    const long long want = std::max<long long>(1024, n * 24);
    if (c->fcap < want) {
        VG_CUDA(ensure(c, c->d_faces, want));
        c->fcap = want;
    }
    VG_CUDA(ensure(c, c->d_rank, n));
    VG_CUDA(ensure(c, c->d_subset, m));
    VG_CUDA(ensure(c, c->d_subset_in, m));
    const int32_t *in = cells;
    if (!on_device && m > 0) {
        VG_CUDA(cudaMemcpyAsync(c->d_subset_in, cells, sizeof(int) * m, cudaMemcpyHostToDevice, c->stream));
        in = c->d_subset_in;
    }
    cudaError_t e = map_cells(c->d_sid, n, in, m, c->d_rank, c->d_subset, c->d_err + 2, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "map_cells");
    int bad = 0;
    VG_CUDA(cudaMemcpyAsync(&bad, c->d_err + 2, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    VG_CUDA(cudaStreamSynchronize(c->stream));
    if (bad) return fail(c, VG_ERR_ARG, std::to_string(bad) + " cell indices outside [0, n)");
    const bool timed = cfg.time_kernels && c->nev < vg_ctx::NEV;
    if (timed) {
        for (int k = 0; k < 2; k++)
            if (!c->ev[2 * c->nev + k]) VG_CUDA(cudaEventCreate(&c->ev[2 * c->nev + k]));
        VG_CUDA(cudaEventRecord(c->ev[2 * c->nev], c->stream));
    }
    e = enqueue_cells(c, cfg, c->stream, c->d_subset, (int)m);
    if (e != cudaSuccess) return cuda_fail(c, e, "cell kernels");
    if (timed) {
        VG_CUDA(cudaEventRecord(c->ev[2 * c->nev + 1], c->stream));
        c->nev++;
    }
    c->launches += g_launch_count - l0;
    c->computed = 1;
    c->wb_valid = 0;
    c->subset = 1;
    return VG_OK;
}

vg_status vg_graph_capture(vg_ctx *c, const int64_t *counts, const void *pos, const void *radii, int dtype,
                           const vg_config *cfg_in) {
    if (!c) return VG_ERR_ARG;
    vg_config cfg;
    if (cfg_in) cfg = *cfg_in; else vg_config_default(&cfg);
    vg_status s = check_config(c, cfg, true);
    if (s != VG_OK) return s;
    if (!counts) return fail(c, VG_ERR_ARG, "counts is NULL");
    std::vector<long long> cv(c->sys.size());
    long long n = 0;
    for (size_t k = 0; k < cv.size(); k++) {
        if (counts[k] < 0) return fail(c, VG_ERR_ARG, "negative particle count");
        cv[k] = counts[k];
        n += cv[k];
    }
    // a replay reads its input from fixed device addresses
    for (const void *p : {pos, radii}) {
        if (!p) continue;
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, VG_ERR_ARG, "graph input is not device memory");
        }
        if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
            return fail(c, VG_ERR_ARG, "graph input is not device memory");
    }
    std::vector<int64_t> keep(counts, counts + cv.size());
    // one eager pass validates the input, sizes every buffer and leaves
    // valid results
    if ((s = insert_all(c, cv, pos, radii, dtype, 1)) != VG_OK) return s;
    vg_config eager = cfg;
    eager.time_kernels = 0;
    if ((s = vg_compute(c, &eager)) != VG_OK) return s;
    unsigned long long used = 0;
    VG_CUDA(cudaMemcpyAsync(&used, c->d_fcount, sizeof used, cudaMemcpyDeviceToHost, c->stream));
    VG_CUDA(cudaStreamSynchronize(c->stream));
    // headroom for inputs that change between replays
    const long long room = (long long)(used * 5 / 4) + 4096;
    if (c->fcap < room) {
        VG_CUDA(ensure(c, c->d_faces, room));
        c->fcap = room;
    }
    if ((s = ensure_csr(c)) != VG_OK) return s;
    if (!c->gstream) VG_CUDA(cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking));
    const bool timed = cfg.time_kernels != 0;
    if (timed)
        for (int k = 0; k < 4; k++)
            if (!c->gev[k]) VG_CUDA(cudaEventCreate(&c->gev[k]));
    const long long l0 = g_launch_count;
    cudaStream_t gs = c->gstream;
    VG_CUDA(cudaStreamBeginCapture(gs, cudaStreamCaptureModeRelaxed));
    cudaError_t e = timed ? cudaEventRecordWithFlags(c->gev[2], gs, cudaEventRecordExternal) : cudaSuccess;
    if (e == cudaSuccess) e = enqueue_sort(c, pos, radii, dtype, gs);
    if (e == cudaSuccess && timed) e = cudaEventRecordWithFlags(c->gev[3], gs, cudaEventRecordExternal);
    if (e == cudaSuccess && timed) e = cudaEventRecordWithFlags(c->gev[0], gs, cudaEventRecordExternal);
    if (e == cudaSuccess) e = enqueue_cells(c, cfg, gs);
    if (e == cudaSuccess && timed) e = cudaEventRecordWithFlags(c->gev[1], gs, cudaEventRecordExternal);
    if (e == cudaSuccess && cfg.weinberg)
        e = launch_weinberg(c->d_topo, c->d_topo_n, c->n, c->d_wlen, c->d_whash, c->d_wsym, c->sm_count, gs);
    if (e == cudaSuccess) e = enqueue_compact(c, gs);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(gs, &g);
    const long long kernels = g_launch_count - l0;
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(c, e, "graph capture");
    }
    c->graph = g;
    e = cudaGraphInstantiate(&c->gexec, g, 0);
    if (e != cudaSuccess) {
        release_graph(c);
        return cuda_fail(c, e, "cudaGraphInstantiate");
    }
    if (timed) {
        size_t nn = 0;
        VG_CUDA(cudaGraphGetNodes(g, nullptr, &nn));
        std::vector<cudaGraphNode_t> nodes(nn);
        VG_CUDA(cudaGraphGetNodes(g, nodes.data(), &nn));
        for (cudaGraphNode_t nd : nodes) {
            cudaGraphNodeType ty;
            VG_CUDA(cudaGraphNodeGetType(nd, &ty));
            if (ty != cudaGraphNodeTypeEventRecord) continue;
            cudaEvent_t ev = nullptr;
            VG_CUDA(cudaGraphEventRecordNodeGetEvent(nd, &ev));
            for (int k = 0; k < 4; k++)
                if (ev == c->gev[k]) c->gev_node[k] = nd;
        }
        if (!c->gev_node[0] || !c->gev_node[1] || !c->gev_node[2] || !c->gev_node[3]) {
            release_graph(c);
            return fail(c, VG_ERR_CUDA, "graph capture lost its timing events");
        }
    }
    c->graph_kernels = kernels;
    c->graph_timed = timed ? 1 : 0;
    c->g_counts = keep;
    c->g_pos = pos;
    c->g_rad = radii;
    c->g_dtype = dtype;
    c->g_cfg = cfg;
    return VG_OK;
}

vg_status vg_graph_launch(vg_ctx *c) {
    if (!c) return VG_ERR_ARG;
    if (!c->gexec) return fail(c, VG_ERR_STATE, "no captured graph");
    if (c->graph_timed && c->nev < vg_ctx::NEV) {
        for (int k = 0; k < 2; k++) {
            cudaEvent_t &ev = c->ev[2 * c->nev + k];
            if (!ev) VG_CUDA(cudaEventCreate(&ev));
            VG_CUDA(cudaGraphExecEventRecordNodeSetEvent(c->gexec, c->gev_node[k], ev));
        }
        c->nev++;
    }
    if (c->graph_timed && c->nsev < vg_ctx::NEV) {
        for (int k = 0; k < 2; k++) {
            cudaEvent_t &ev = c->sev[2 * c->nsev + k];
            if (!ev) VG_CUDA(cudaEventCreate(&ev));
            VG_CUDA(cudaGraphExecEventRecordNodeSetEvent(c->gexec, c->gev_node[2 + k], ev));
        }
        c->nsev++;
    }
    VG_CUDA(cudaGraphLaunch(c->gexec, c->stream));
    c->launches += c->graph_kernels;
    c->inserted = 1;
    c->computed = 1;
    c->wb_valid = c->g_cfg.weinberg ? 1 : 0;
    c->subset = 0;
    c->graph_unchecked = 1;
    if (c->pred) c->kblock_valid = 1;
    return VG_OK;
}

vg_status vg_graph_sync(vg_ctx *c) {
    if (!c) return VG_ERR_ARG;
    if (!c->graph_unchecked) {
        VG_CUDA(cudaStreamSynchronize(c->stream));
        return VG_OK;
    }
    return graph_check(c);
}

vg_status vg_get_counts(vg_ctx *c, int64_t *n_cells, int64_t *n_faces) {
    if (!c) return VG_ERR_ARG;
    if (c->graph_unchecked) {
        vg_status gs = graph_check(c);
        if (gs != VG_OK) return gs;
    }
    if (!c->computed) return fail(c, VG_ERR_STATE, "no computed cells");
    if (c->subset) return fail(c, VG_ERR_STATE, "faces exist after a full compute only");
    if (n_cells) *n_cells = c->n;
    if (n_faces) {
        long long t = 0;
        VG_CUDA(cudaMemcpyAsync(&t, c->d_face_off + c->n, sizeof t, cudaMemcpyDeviceToHost, c->stream));
        VG_CUDA(cudaStreamSynchronize(c->stream));
        *n_faces = t;
    }
    return VG_OK;
}

vg_status vg_get_cells(vg_ctx *c, double *vol, double *area, double *centroid, int32_t *nv, int32_t *ne,
                       int32_t *nf, uint8_t *status, int on_device) {
    if (!c) return VG_ERR_ARG;
    if (c->graph_unchecked) {
        vg_status gs = graph_check(c);
        if (gs != VG_OK) return gs;
    }
    if (!c->computed) return fail(c, VG_ERR_STATE, "no computed cells");
    const long long n = c->n;
    vg_status s;
    if ((s = copy_out(c, vol, c->d_vol, sizeof(double) * n, on_device))) return s;
    if ((s = copy_out(c, area, c->d_area, sizeof(double) * n, on_device))) return s;
    if (centroid) {
        if (c->dim == 3) {
            if ((s = copy_out(c, centroid, c->d_cen, sizeof(double) * n * 3, on_device))) return s;
        } else if (n > 0) {
            // stored with stride 3; pack to n x 2
            VG_CUDA(cudaMemcpy2DAsync(centroid, 2 * sizeof(double), c->d_cen, 3 * sizeof(double), 2 * sizeof(double),
                                      n, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
            if (!on_device) VG_CUDA(cudaStreamSynchronize(c->stream));
        }
    }
    if ((s = copy_out(c, nv, c->d_nv, sizeof(int) * n, on_device))) return s;
    if ((s = copy_out(c, ne, c->d_ne, sizeof(int) * n, on_device))) return s;
    if ((s = copy_out(c, nf, c->d_nf, sizeof(int) * n, on_device))) return s;
    if ((s = copy_out(c, status, c->d_status, n, on_device))) return s;
    return VG_OK;
}

vg_status vg_get_faces(vg_ctx *c, int64_t *face_off, int32_t *nbr_id, int8_t *nbr_img, uint8_t *face_order,
                       int on_device) {
    if (!c) return VG_ERR_ARG;
    if (c->graph_unchecked) {
        vg_status gs = graph_check(c);
        if (gs != VG_OK) return gs;
    }
    if (!c->computed) return fail(c, VG_ERR_STATE, "no computed cells");
    if (c->subset) return fail(c, VG_ERR_STATE, "faces exist after a full compute only");
    const long long n = c->n;
    long long t = 0;
    VG_CUDA(cudaMemcpyAsync(&t, c->d_face_off + n, sizeof t, cudaMemcpyDeviceToHost, c->stream));
    VG_CUDA(cudaStreamSynchronize(c->stream));
    vg_status s;
    if ((s = copy_out(c, face_off, c->d_face_off, sizeof(long long) * (n + 1), on_device))) return s;
    if ((s = copy_out(c, nbr_id, c->d_nbr, sizeof(int) * t, on_device))) return s;
    if ((s = copy_out(c, nbr_img, c->d_img, 3 * (size_t)t, on_device))) return s;
    if ((s = copy_out(c, face_order, c->d_ford, (size_t)t, on_device))) return s;
    return VG_OK;
}

vg_status vg_get_kernel_ms(vg_ctx *c, double *total_ms, int64_t *count) {
    if (!c || !total_ms || !count) return VG_ERR_ARG;
    VG_CUDA(cudaStreamSynchronize(c->stream));
    double t = 0;
    for (int k = 0; k < c->nev; k++) {
        float ms = 0;
        VG_CUDA(cudaEventElapsedTime(&ms, c->ev[2 * k], c->ev[2 * k + 1]));
        t += ms;
    }
    *total_ms = t;
    *count = c->nev;
    c->nev = 0;
    return VG_OK;
}

vg_status vg_get_sort_ms(vg_ctx *c, double *total_ms, int64_t *count) {
    if (!c || !total_ms || !count) return VG_ERR_ARG;
    VG_CUDA(cudaStreamSynchronize(c->stream));
    double t = 0;
    for (int k = 0; k < c->nsev; k++) {
        float ms = 0;
        VG_CUDA(cudaEventElapsedTime(&ms, c->sev[2 * k], c->sev[2 * k + 1]));
        t += ms;
    }
    *total_ms = t;
    *count = c->nsev;
    c->nsev = 0;
    return VG_OK;
}

vg_status vg_set_system_split(vg_ctx *c, int k, int split) {
    if (!c || k < 0 || k >= (int)c->sys.size() || (split != 0 && split != 1)) return VG_ERR_ARG;
    c->sys[k].hot = split;
    // both device copies: the descriptor each insert starts from and the one
    // the cell kernels read (a captured graph reads them at every replay)
    const size_t at = sizeof(Sys) * (size_t)k + offsetof(Sys, hot);
    for (Sys *d : {c->d_sys_init, c->d_sys}) {
        if (!d) continue;
        VG_CUDA(cudaMemcpyAsync(reinterpret_cast<char *>(d) + at, &c->sys[k].hot, sizeof(int),
                                cudaMemcpyHostToDevice, c->stream));
    }
    VG_CUDA(cudaStreamSynchronize(c->stream));
    return VG_OK;
}

vg_status vg_get_deferred(vg_ctx *c, int64_t *count) {
    if (!c || !count) return VG_ERR_ARG;
    if (!c->computed) return fail(c, VG_ERR_STATE, "no computed cells");
    int k = 0;
    VG_CUDA(cudaMemcpyAsync(&k, c->d_capcount0, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    VG_CUDA(cudaStreamSynchronize(c->stream));
    *count = k;
    return VG_OK;
}

vg_status vg_get_work(vg_ctx *c, int32_t *n_tested, int32_t *n_vtests, int32_t *n_cuts, int32_t *n_newv,
                      int32_t *n_retest, uint8_t *fallback, int32_t *n_prefetch, int on_device) {
    if (!c) return VG_ERR_ARG;
    if (c->graph_unchecked) {
        vg_status gs = graph_check(c);
        if (gs != VG_OK) return gs;
    }
    if (!c->computed) return fail(c, VG_ERR_STATE, "no computed cells");
    const long long n = c->n;
    vg_status s;
    if ((s = copy_out(c, n_tested, c->d_w_tested, sizeof(int) * n, on_device))) return s;
    if ((s = copy_out(c, n_vtests, c->d_w_vtests, sizeof(int) * n, on_device))) return s;
    if ((s = copy_out(c, n_cuts, c->d_w_cuts, sizeof(int) * n, on_device))) return s;
    if ((s = copy_out(c, n_newv, c->d_w_newv, sizeof(int) * n, on_device))) return s;
    if ((s = copy_out(c, n_retest, c->d_w_retest, sizeof(int) * n, on_device))) return s;
    if ((s = copy_out(c, fallback, c->d_w_fallback, n, on_device))) return s;
    if ((s = copy_out(c, n_prefetch, c->d_w_pref, sizeof(int) * n, on_device))) return s;
    return VG_OK;
}

vg_status vg_get_radius(vg_ctx *c, float *rmax, int on_device) {
    if (!c) return VG_ERR_ARG;
    if (c->graph_unchecked) {
        vg_status gs = graph_check(c);
        if (gs != VG_OK) return gs;
    }
    if (!c->computed) return fail(c, VG_ERR_STATE, "no computed cells");
    return copy_out(c, rmax, c->d_rfin, sizeof(float) * c->n, on_device);
}

vg_status vg_get_weinberg(vg_ctx *c, int32_t *len, uint64_t *hash, int32_t *sym, int on_device) {
    if (!c) return VG_ERR_ARG;
    if (c->graph_unchecked) {
        vg_status gs = graph_check(c);
        if (gs != VG_OK) return gs;
    }
    if (!c->computed) return fail(c, VG_ERR_STATE, "no computed cells");
    if (!c->wb_valid) return fail(c, VG_ERR_STATE, "no Weinberg codes: compute with cfg.weinberg = 1");
    vg_status s;
    if ((s = copy_out(c, len, c->d_wlen, sizeof(int) * c->n, on_device))) return s;
    if ((s = copy_out(c, hash, c->d_whash, sizeof(unsigned long long) * c->n, on_device))) return s;
    return copy_out(c, sym, c->d_wsym, sizeof(int) * c->n, on_device);
}

vg_status vg_get_sorted(vg_ctx *c, int64_t *n_blocks, int32_t *block_start, int32_t *order, int on_device) {
    if (!c) return VG_ERR_ARG;
    if (c->graph_unchecked) {
        vg_status gs = graph_check(c);
        if (gs != VG_OK) return gs;
    }
    if (!c->inserted) return fail(c, VG_ERR_STATE, "nothing inserted");
    if (n_blocks) *n_blocks = c->total_blk;
    vg_status s;
    if ((s = copy_out(c, block_start, c->d_bstart, sizeof(int) * (c->total_blk + 1), on_device))) return s;
    if ((s = copy_out(c, order, c->d_sid, sizeof(int) * c->n, on_device))) return s;
    return VG_OK;
}

vg_status vg_get_launches(vg_ctx *c, int64_t *count) {
    if (!c || !count) return VG_ERR_ARG;
    *count = c->launches;
    return VG_OK;
}

vg_status vg_get_grid(vg_ctx *c, int *nblocks) {
    if (!c || !nblocks) return VG_ERR_ARG;
    for (int a = 0; a < c->dim; a++) nblocks[a] = c->sys[0].g.nb[a];
    return VG_OK;
}

vg_status vg_get_system_grid(vg_ctx *c, int k, int *nblocks) {
    if (!c || !nblocks || k < 0 || k >= (int)c->sys.size()) return VG_ERR_ARG;
    for (int a = 0; a < c->dim; a++) nblocks[a] = c->sys[k].g.nb[a];
    return VG_OK;
}

const char *vg_last_error(vg_ctx *c) { return c ? c->err.c_str() : "null context"; }

void vg_destroy(vg_ctx *c) {
    if (!c) return;
    release(c->d_pos); release(c->d_rad); release(c->d_pos32); release(c->d_rad32); release(c->d_key); release(c->d_slot); release(c->d_tmp);
    release(c->d_p32); release(c->d_p64); release(c->d_sid); release(c->d_sblk); release(c->d_ssys);
    release(c->d_count); release(c->d_bstart); release(c->d_err); release(c->d_sys);
    if (c->d_scan) cudaFree(c->d_scan);
    release(c->d_vol); release(c->d_area); release(c->d_cen); release(c->d_nv); release(c->d_ne);
    release(c->d_nf); release(c->d_status); release(c->d_fptr); release(c->d_faces); release(c->d_fcount);
    release(c->d_ticket); release(c->d_face_off); release(c->d_nbr); release(c->d_img); release(c->d_ford);
    release(c->d_w_tested); release(c->d_w_vtests); release(c->d_w_cuts); release(c->d_w_retest);
    release(c->d_w_fallback); release(c->d_caplist); release(c->d_capcount);
    release(c->d_caplist2); release(c->d_capcount2); release(c->d_caplist0); release(c->d_capcount0);
    release(c->d_off_code); release(c->d_off_lb); release(c->d_kblock); release(c->d_rho); release(c->d_w_newv);
    release(c->d_w_pref); release(c->d_rfin);
    release(c->d_topo); release(c->d_topo_n); release(c->d_wlen); release(c->d_wsym); release(c->d_whash);
    release(c->d_kstar); release(c->d_kmax); release(c->d_feat);
    release(c->d_rank); release(c->d_subset); release(c->d_subset_in);
    release(c->d_sys_init);
    release_graph(c);
    for (int k = 0; k < 4; k++)
        if (c->gev[k]) cudaEventDestroy(c->gev[k]);
    if (c->gstream) cudaStreamDestroy(c->gstream);
    for (int k = 0; k < 2 * vg_ctx::NEV; k++) {
        if (c->ev[k]) cudaEventDestroy(c->ev[k]);
        if (c->sev[k]) cudaEventDestroy(c->sev[k]);
    }
    delete c;
}

}  // extern "C"

namespace {

// Reads what a replay flagged: input errors, and a face buffer too small for
// this replay's input -- then the step is redone eagerly (which grows the
// buffer) and the graph re-captured, so the results are complete.
vg_status graph_check(vg_ctx *c) {
    c->graph_unchecked = 0;
    vg_status s = read_input_flags(c);
    if (s != VG_OK) {
        c->computed = 0;
        c->wb_valid = 0;
        return s;
    }
    unsigned long long used = 0;
    VG_CUDA(cudaMemcpyAsync(&used, c->d_fcount, sizeof used, cudaMemcpyDeviceToHost, c->stream));
    VG_CUDA(cudaStreamSynchronize(c->stream));
    if ((long long)used <= c->fcap) return VG_OK;
    const std::vector<int64_t> counts = c->g_counts;
    const vg_config cfg = c->g_cfg;
    return vg_graph_capture(c, counts.data(), c->g_pos, c->g_rad, c->g_dtype, &cfg);
}

}  // namespace
