// Host side of the C ABI declared in include/vorogpu.h: argument checks,
// device buffers, the sort -> cells -> faces pipeline, and result copies.
#include <math.h>
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

#define VG_CUDA(call)                                       \
    do {                                                    \
        cudaError_t e_ = (call);                            \
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
void grid_from_nopt(vg_ctx *c, long long n) {
    double V = 1;
    for (int a = 0; a < c->dim; a++) V *= c->g.L[a];
    double nopt = c->n_opt > 0 ? c->n_opt : (c->dim == 3 ? 4.6 : 3.4);
    double lam = pow((double)std::max<long long>(n, 1) / (nopt * V), 1.0 / c->dim);
    for (int a = 0; a < c->dim; a++) {
        long long v = (long long)floor(lam * c->g.L[a]);
        c->g.nb[a] = (int)std::max<long long>(1, std::min<long long>(v, 1 << 20));
    }
}

void finish_grid(vg_ctx *c) {
    Grid &g = c->g;
    g.nblk = 1;
    for (int a = 0; a < 3; a++) {
        if (a >= c->dim) { g.nb[a] = 1; g.lo[a] = 0; g.hi[a] = 1; g.L[a] = 1; g.per[a] = 0; }
        g.h[a] = g.L[a] / g.nb[a];
        g.hf[a] = (float)g.h[a];
        g.Lf[a] = (float)g.L[a];
        g.nblk *= g.nb[a];
    }
}

// Sorted list of block offsets for the walk: all offsets whose distance
// bound from the home block lies below shell * h_min, ascending.
vg_status build_offsets(vg_ctx *c) {
    const Grid &g = c->g;
    int S = 4;
    double hmin = 1e300;
    for (int a = 0; a < c->dim; a++) hmin = std::min(hmin, g.h[a]);
    struct E { float lb; int l1; int code; };
    std::vector<E> v;
    int lim[3];
    for (int a = 0; a < 3; a++) lim[a] = a < c->dim ? S : 0;
    for (int z = -lim[2]; z <= lim[2]; z++)
        for (int y = -lim[1]; y <= lim[1]; y++)
            for (int x = -lim[0]; x <= lim[0]; x++) {
                int o[3] = {x, y, z};
                double lb2 = 0;
                for (int a = 0; a < 3; a++) {
                    double t = std::max(0, std::abs(o[a]) - 1) * (double)g.hf[a];
                    lb2 += t * t;
                }
                float lb = (float)sqrt(lb2);
                // the kernel's shell continuation skips offsets whose FP32
                // bound is below shell*h_min; keep exactly those here
                float lbx = fmaxf(0.f, (float)(std::abs(x) - 1)) * g.hf[0];
                float lby = fmaxf(0.f, (float)(std::abs(y) - 1)) * g.hf[1];
                float lbz = fmaxf(0.f, (float)(std::abs(z) - 1)) * g.hf[2];
                float lbmax = (float)S * (float)hmin;
                if (!(lbx * lbx + lby * lby + lbz * lbz < lbmax * lbmax)) continue;
                int code = (x & 0xff) | ((y & 0xff) << 8) | ((z & 0xff) << 16);
                v.push_back({lb, std::abs(x) + std::abs(y) + std::abs(z), code});
            }
    std::stable_sort(v.begin(), v.end(), [](const E &a, const E &b) {
        if (a.lb != b.lb) return a.lb < b.lb;
        return a.l1 < b.l1;
    });
    std::vector<int> code(v.size());
    std::vector<float> lb(v.size());
    for (size_t i = 0; i < v.size(); i++) { code[i] = v[i].code; lb[i] = v[i].lb; }
    release(c->d_off_code);
    release(c->d_off_lb);
    VG_CUDA(cudaMalloc((void **)&c->d_off_code, sizeof(int) * code.size()));
    VG_CUDA(cudaMalloc((void **)&c->d_off_lb, sizeof(float) * lb.size()));
    VG_CUDA(cudaMemcpy(c->d_off_code, code.data(), sizeof(int) * code.size(), cudaMemcpyHostToDevice));
    VG_CUDA(cudaMemcpy(c->d_off_lb, lb.data(), sizeof(float) * lb.size(), cudaMemcpyHostToDevice));
    c->off_count = (int)code.size();
    c->off_shell = S;
    return VG_OK;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
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
    cfg->prefetch_k = 0;
    cfg->use_mlp = 0;
    cfg->chunk = 0;
    cfg->warps_per_cta = 0;
    cfg->collect_stats = 0;
    cfg->time_kernels = 0;
}

vg_status vg_create(vg_ctx **out, int dim, const double *lo, const double *hi, const int *periodic,
                    const int *nblocks, double n_opt, void *stream) {
    if (!out) return VG_ERR_ARG;
    *out = nullptr;
    if (dim != 2 && dim != 3) return VG_ERR_ARG;
    if (!lo || !hi || !periodic) return VG_ERR_ARG;
    vg_ctx *c = new (std::nothrow) vg_ctx();
    if (!c) return VG_ERR_OOM;
    c->dim = dim;
    c->g.dim = dim;
    for (int a = 0; a < dim; a++) {
        if (!isfinite(lo[a]) || !isfinite(hi[a]) || !(hi[a] > lo[a])) {
            delete c;
            return VG_ERR_ARG;
        }
        c->g.lo[a] = lo[a];
        c->g.hi[a] = hi[a];
        c->g.L[a] = hi[a] - lo[a];
        c->g.per[a] = periodic[a] ? 1 : 0;
        c->g.nb[a] = 1;
    }
    if (nblocks) {
        for (int a = 0; a < dim; a++) {
            if (nblocks[a] < 1 || nblocks[a] > (1 << 20)) { delete c; return VG_ERR_ARG; }
            c->g.nb[a] = nblocks[a];
        }
        long long prod = 1;
        for (int a = 0; a < dim; a++) prod *= nblocks[a];
        if (prod > (1ll << 30)) { delete c; return VG_ERR_ARG; }
        c->grid_fixed = 1;
    }
    c->n_opt = n_opt;
    c->stream = (cudaStream_t)stream;
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return VG_ERR_CUDA;
    }
    finish_grid(c);
    if (build_offsets(c) != VG_OK) { vg_destroy(c); return VG_ERR_CUDA; }
    VG_CUDA(cudaMalloc((void **)&c->d_err, sizeof(int) * 4));
    VG_CUDA(cudaMalloc((void **)&c->d_fcount, sizeof(unsigned long long)));
    VG_CUDA(cudaMalloc((void **)&c->d_ticket, sizeof(unsigned) * 4));
    VG_CUDA(cudaMalloc((void **)&c->d_capcount, sizeof(int)));
    VG_CUDA(cudaMalloc((void **)&c->d_capcount2, sizeof(int)));
    *out = c;
    return VG_OK;
}

vg_status vg_insert(vg_ctx *c, int64_t n, const double *pos, const double *radii, int on_device) {
    if (!c) return VG_ERR_ARG;
    if (n < 0 || n > 0x7ffffffe) return fail(c, VG_ERR_ARG, "particle count out of range");
    if (n > 0 && !pos) return fail(c, VG_ERR_ARG, "pos is NULL");
    c->inserted = 0;
    c->computed = 0;
    const int d = c->dim;
    if (!c->grid_fixed) {
        grid_from_nopt(c, n);
        finish_grid(c);
        vg_status s = build_offsets(c);
        if (s != VG_OK) return s;
    }
    double V = 1;
    for (int a = 0; a < d; a++) V *= c->g.L[a];
    c->g.s = pow(V / (double)std::max<int64_t>(n, 1), 1.0 / d);
    VG_CUDA(ensure(c, c->d_key, n));
    VG_CUDA(ensure(c, c->d_slot, n));
    VG_CUDA(ensure(c, c->d_tmp, n));
    VG_CUDA(ensure(c, c->d_p32, n));
    VG_CUDA(ensure(c, c->d_p64, n));
    VG_CUDA(ensure(c, c->d_sid, n));
    VG_CUDA(ensure(c, c->d_sblk, n));
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
    VG_CUDA(ensure(c, c->d_w_tested, n));
    VG_CUDA(ensure(c, c->d_w_vtests, n));
    VG_CUDA(ensure(c, c->d_w_cuts, n));
    VG_CUDA(ensure(c, c->d_w_retest, n));
    VG_CUDA(ensure(c, c->d_w_newv, n));
    VG_CUDA(ensure(c, c->d_w_fallback, n));
    if (!on_device) {
        VG_CUDA(ensure(c, c->d_pos, n * d));
        if (radii) VG_CUDA(ensure(c, c->d_rad, n));
    }
    VG_CUDA(ensure(c, c->d_count, c->g.nblk));
    VG_CUDA(ensure(c, c->d_bstart, c->g.nblk + 1));
    size_t need_scan = std::max(scan_tmp_bytes_i32(c->g.nblk + 1),
                                (((size_t)n * sizeof(int) + 255) & ~(size_t)255) + scan_tmp_bytes_i64(n + 1));
    if (need_scan > c->scan_bytes) {
        if (c->d_scan) cudaFree(c->d_scan);
        c->d_scan = nullptr;
        c->scan_bytes = 0;
        VG_CUDA(cudaMalloc(&c->d_scan, need_scan));
        c->scan_bytes = need_scan;
    }
    const double *dpos = pos, *drad = radii;
    if (n > 0 && !on_device) {
        VG_CUDA(cudaMemcpyAsync(c->d_pos, pos, sizeof(double) * n * d, cudaMemcpyHostToDevice, c->stream));
        dpos = c->d_pos;
        if (radii) {
            VG_CUDA(cudaMemcpyAsync(c->d_rad, radii, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
            drad = c->d_rad;
        }
    }
    c->n = n;
    c->radical = radii != nullptr;
    c->rmax = 0;
    if (radii) {
        // the radical stop test needs the largest radius
        std::vector<double> hr;
        const double *src = radii;
        if (on_device) {
            hr.resize((size_t)n);
            VG_CUDA(cudaMemcpyAsync(hr.data(), radii, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
            VG_CUDA(cudaStreamSynchronize(c->stream));
            src = hr.data();
        }
        for (int64_t i = 0; i < n; i++) if (src[i] > c->rmax) c->rmax = src[i];
    }
    const long long l0 = g_launch_count;
    cudaError_t e = sort_particles(c->g, n, dpos, drad, c->d_key, c->d_slot, c->d_count, c->d_bstart,
                                   c->d_tmp, c->d_p32, c->d_p64, c->d_sid, c->d_sblk, c->d_err,
                                   c->d_scan, c->scan_bytes, c->stream);
    c->launches += g_launch_count - l0;
    if (e != cudaSuccess) return cuda_fail(c, e, "sort_particles");
    int herr[2] = {0, 0};
    VG_CUDA(cudaMemcpyAsync(herr, c->d_err, sizeof(int) * 2, cudaMemcpyDeviceToHost, c->stream));
    VG_CUDA(cudaStreamSynchronize(c->stream));
    if (herr[1]) return fail(c, VG_ERR_NONFINITE, std::to_string(herr[1]) + " non-finite coordinates or radii");
    if (herr[0]) return fail(c, VG_ERR_OUT_OF_BOX, std::to_string(herr[0]) + " particles outside a walled box");
    c->inserted = 1;
    return VG_OK;
}

vg_status vg_compute(vg_ctx *c, const vg_config *cfg_in) {
    if (!c) return VG_ERR_ARG;
    if (!c->inserted) return fail(c, VG_ERR_STATE, "vg_compute before vg_insert");
    vg_config cfg;
    if (cfg_in) cfg = *cfg_in; else vg_config_default(&cfg);
    if (cfg.precision != VG_FP64 && cfg.precision != VG_FP32_RETEST) return fail(c, VG_ERR_ARG, "precision");
    if (cfg.order != VG_WALK && cfg.order != VG_PREFETCH) return fail(c, VG_ERR_ARG, "order");
    if (!(cfg.tol32 > 0) || !(cfg.tau_rel > 0) || !(cfg.merge_rel > 0)) return fail(c, VG_ERR_ARG, "tolerances");
    if (cfg.use_mlp && !c->d_kblock) return fail(c, VG_ERR_STATE, "use_mlp without MLP predictions");
    const long long n = c->n;
    const long long l0 = g_launch_count;
    // face buffer: start at 24 faces per cell, grow on overflow
    long long want = std::max<long long>(1024, n * 24);
    if (c->fcap < want) {
        VG_CUDA(ensure(c, c->d_faces, want));
        c->fcap = want;
    }
    Store st;
    st.p32 = c->d_p32; st.p64 = c->d_p64; st.sid = c->d_sid; st.sblk = c->d_sblk; st.bstart = c->d_bstart;
    st.n = (int)n; st.radical = c->radical; st.rmax = c->rmax;
    Params pp;
    pp.tol32 = cfg.tol32; pp.tau_rel = cfg.tau_rel; pp.merge_rel = cfg.merge_rel;
    pp.prefetch_k = cfg.prefetch_k; pp.order = cfg.order;
    pp.chunk = cfg.chunk > 0 ? cfg.chunk : 2;
    pp.collect = cfg.collect_stats ? 1 : 0;
    pp.kblock = cfg.use_mlp ? c->d_kblock : nullptr;
    Offsets off;
    off.code = c->d_off_code; off.lb = c->d_off_lb; off.count = c->off_count; off.shell = c->off_shell;
    for (int attempt = 0; attempt < 4; attempt++) {
        Out o;
        o.vol = c->d_vol; o.area = c->d_area; o.cen = c->d_cen;
        o.nv = c->d_nv; o.ne = c->d_ne; o.nf = c->d_nf; o.status = c->d_status;
        o.fptr = c->d_fptr; o.faces = c->d_faces; o.fcount = c->d_fcount; o.fcap = c->fcap;
        o.w_tested = c->d_w_tested; o.w_vtests = c->d_w_vtests; o.w_cuts = c->d_w_cuts;
        o.w_retest = c->d_w_retest; o.w_fallback = c->d_w_fallback; o.w_newv = c->d_w_newv;
        o.retry = c->d_caplist; o.retry_count = c->d_capcount;
        o.retry2 = c->d_caplist2; o.retry2_count = c->d_capcount2;
        VG_CUDA(cudaMemsetAsync(c->d_fcount, 0, sizeof(unsigned long long), c->stream));
        VG_CUDA(cudaMemsetAsync(c->d_capcount, 0, sizeof(int), c->stream));
        VG_CUDA(cudaMemsetAsync(c->d_capcount2, 0, sizeof(int), c->stream));
        cudaError_t e;
        const bool timed = cfg.time_kernels && c->nev < vg_ctx::NEV;
        if (timed) {
            for (int k = 0; k < 2; k++)
                if (!c->ev[2 * c->nev + k]) VG_CUDA(cudaEventCreate(&c->ev[2 * c->nev + k]));
            VG_CUDA(cudaEventRecord(c->ev[2 * c->nev], c->stream));
        }
        if (c->dim == 3) {
            e = launch_cells3(c->g, st, o, pp, off, cfg.precision, c->d_ticket, c->sm_count, cfg.warps_per_cta,
                              nullptr, (int)n, 0, c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "launch_cells3");
            e = launch_cells3(c->g, st, o, pp, off, cfg.precision, c->d_ticket + 1, c->sm_count, 0,
                              c->d_caplist, 0, 1, c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "launch_cells3 (big cells)");
            e = launch_cells3(c->g, st, o, pp, off, cfg.precision, c->d_ticket + 2, c->sm_count, 0,
                              c->d_caplist2, 0, 2, c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "launch_cells3 (largest cells)");
        } else {
            e = launch_cells2(c->g, st, o, pp, off, cfg.precision, c->d_ticket, c->sm_count, cfg.warps_per_cta,
                              nullptr, (int)n, 0, c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "launch_cells2");
            e = launch_cells2(c->g, st, o, pp, off, cfg.precision, c->d_ticket + 1, c->sm_count, 0,
                              c->d_caplist, 0, 1, c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "launch_cells2 (big cells)");
            e = launch_cells2(c->g, st, o, pp, off, cfg.precision, c->d_ticket + 2, c->sm_count, 0,
                              c->d_caplist2, 0, 2, c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "launch_cells2 (largest cells)");
        }
        if (timed) {
            VG_CUDA(cudaEventRecord(c->ev[2 * c->nev + 1], c->stream));
            c->nev++;
        }
        unsigned long long used = 0;
        VG_CUDA(cudaMemcpyAsync(&used, c->d_fcount, sizeof used, cudaMemcpyDeviceToHost, c->stream));
        VG_CUDA(cudaStreamSynchronize(c->stream));
        if ((long long)used <= c->fcap) {
            c->total_faces = -1;
            break;
        }
        // face buffer too small: grow to what was asked for and recompute
        long long need = (long long)(used * 5 / 4) + 1024;
        VG_CUDA(ensure(c, c->d_faces, need));
        c->fcap = need;
        if (attempt == 3) return fail(c, VG_ERR_CAP, "face buffer overflow");
    }
    // CSR of faces
    long long need_csr = c->fcap;
    VG_CUDA(ensure(c, c->d_nbr, need_csr));
    VG_CUDA(ensure(c, c->d_img, 3 * need_csr));
    VG_CUDA(ensure(c, c->d_ford, need_csr));
    cudaError_t e = compact_faces(n, c->d_nf, c->d_status, c->d_fptr, c->d_faces, c->d_face_off, c->d_nbr,
                                  c->d_img, c->d_ford, c->d_scan, c->stream);
    c->launches += g_launch_count - l0;
    if (e != cudaSuccess) return cuda_fail(c, e, "compact_faces");
    c->computed = 1;
    c->total_faces = -1;
    return VG_OK;
}

vg_status vg_get_counts(vg_ctx *c, int64_t *n_cells, int64_t *n_faces) {
    if (!c) return VG_ERR_ARG;
    if (!c->computed) return fail(c, VG_ERR_STATE, "no computed cells");
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
    if (!c->computed) return fail(c, VG_ERR_STATE, "no computed cells");
    const long long n = c->n;
    vg_status s;
    if ((s = copy_out(c, vol, c->d_vol, sizeof(double) * n, on_device))) return s;
    if ((s = copy_out(c, area, c->d_area, sizeof(double) * n, on_device))) return s;
    if (centroid) {
        if (c->dim == 3) {
            if ((s = copy_out(c, centroid, c->d_cen, sizeof(double) * n * 3, on_device))) return s;
        } else {
            // stored with stride 3; pack to n x 2
            VG_CUDA(cudaMemcpy2DAsync(centroid, 2 * sizeof(double), c->d_cen, 3 * sizeof(double),
                                      2 * sizeof(double), n, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                      c->stream));
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
    if (!c->computed) return fail(c, VG_ERR_STATE, "no computed cells");
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

vg_status vg_get_work(vg_ctx *c, int32_t *n_tested, int32_t *n_vtests, int32_t *n_cuts, int32_t *n_newv,
                      int32_t *n_retest, uint8_t *fallback, int on_device) {
    if (!c) return VG_ERR_ARG;
    if (!c->computed) return fail(c, VG_ERR_STATE, "no computed cells");
    const long long n = c->n;
    vg_status s;
    if ((s = copy_out(c, n_tested, c->d_w_tested, sizeof(int) * n, on_device))) return s;
    if ((s = copy_out(c, n_vtests, c->d_w_vtests, sizeof(int) * n, on_device))) return s;
    if ((s = copy_out(c, n_cuts, c->d_w_cuts, sizeof(int) * n, on_device))) return s;
    if ((s = copy_out(c, n_newv, c->d_w_newv, sizeof(int) * n, on_device))) return s;
    if ((s = copy_out(c, n_retest, c->d_w_retest, sizeof(int) * n, on_device))) return s;
    if ((s = copy_out(c, fallback, c->d_w_fallback, n, on_device))) return s;
    return VG_OK;
}

vg_status vg_get_sorted(vg_ctx *c, int64_t *n_blocks, int32_t *block_start, int32_t *order, int on_device) {
    if (!c) return VG_ERR_ARG;
    if (!c->inserted) return fail(c, VG_ERR_STATE, "nothing inserted");
    if (n_blocks) *n_blocks = c->g.nblk;
    vg_status s;
    if ((s = copy_out(c, block_start, c->d_bstart, sizeof(int) * (c->g.nblk + 1), on_device))) return s;
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
    for (int a = 0; a < c->dim; a++) nblocks[a] = c->g.nb[a];
    return VG_OK;
}

const char *vg_last_error(vg_ctx *c) { return c ? c->err.c_str() : "null context"; }

void vg_destroy(vg_ctx *c) {
    if (!c) return;
    release(c->d_pos); release(c->d_rad); release(c->d_key); release(c->d_slot); release(c->d_tmp);
    release(c->d_p32); release(c->d_p64); release(c->d_sid); release(c->d_sblk); release(c->d_count);
    release(c->d_bstart); release(c->d_err);
    if (c->d_scan) cudaFree(c->d_scan);
    release(c->d_vol); release(c->d_area); release(c->d_cen); release(c->d_nv); release(c->d_ne);
    release(c->d_nf); release(c->d_status); release(c->d_fptr); release(c->d_faces); release(c->d_fcount);
    release(c->d_ticket); release(c->d_face_off); release(c->d_nbr); release(c->d_img); release(c->d_ford);
    release(c->d_w_tested); release(c->d_w_vtests); release(c->d_w_cuts); release(c->d_w_retest);
    release(c->d_w_fallback); release(c->d_caplist); release(c->d_capcount);
    release(c->d_caplist2); release(c->d_capcount2);
    release(c->d_off_code); release(c->d_off_lb); release(c->d_kblock); release(c->d_w_newv);
    for (int k = 0; k < 2 * vg_ctx::NEV; k++)
        if (c->ev[k]) cudaEventDestroy(c->ev[k]);
    delete c;
}

}  // extern "C"
