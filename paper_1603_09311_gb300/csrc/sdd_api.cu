// C ABI of libsdd: argument checks, model upload, work-item planning, the
// persistent walk launch and the fixed-order per-node reduction.
#include <cmath>
#include <complex>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/sdd.h"
#include "sdd_internal.cuh"

using namespace sdd;

namespace {

thread_local std::string g_last_error;

sdd_status fail(sdd_status s, const std::string &msg) {
    g_last_error = msg;
    return s;
}

sdd_status cuda_fail(cudaError_t e, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return SDD_E_CUDA;
}

#define SDD_CUDA(call)                                               \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);          \
    } while (0)

// A growable device buffer owned by a context.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaError_t ensure(size_t need) {
        if (need <= bytes) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        size_t want = need + need / 4 + 256;
        cudaError_t e = cudaMalloc(&p, want);
        if (e == cudaSuccess) bytes = want;
        return e;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
};

}  // namespace

struct sdd_ctx {
    int device = 0;
    int n_sm = 0;
    ModelDev M;
    int K = 0, E = 0;
    int geo = GEO_SHAPES;
    DevBuf raster;
    // per-call scratch
    DevBuf items, slots, trunc, counters, queue, err, nodes, node_ids, mean, se;
    DevBuf rec_steps, rec_counts, rec_exit, rec_wall, rec_mlast;
    Item *h_items = nullptr;  // pinned staging of the item table
    size_t h_items_cap = 0;
    cudaEvent_t items_done = nullptr;  // last copy out of h_items finished
    cudaStream_t stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // the item table last uploaded (reused when a call plans the same items)
    std::vector<int64_t> plan_paths;
    int plan_chunk = -1;
    uint32_t plan_offset = 0;
    bool plan_valid = false;
    uint64_t last_h2d = 0;
};

namespace {

// Cap on the steps of one walk: keeps the occupation power sums (up to
// 27 x steps for four materials) inside 32 bits.
constexpr int64_t kMaxSteps = 1ll << 26;

int kmax_for(int K) { return K <= 2 ? 2 : (K <= 3 ? 3 : (K <= 4 ? 4 : 8)); }

std::complex<double> column_value(double kappa, double z) {
    const std::complex<double> k = std::sqrt(std::complex<double>(0.0, kappa));
    if (z >= 0.0) return std::exp(-k * z);
    return 1.0 - k * z;
}

sdd_status check_model(const sdd_model_desc *m) {
    if (!m) return fail(SDD_E_ARG, "model is NULL");
    const sdd_domain &d = m->domain;
    if (!(std::isfinite(d.x_min) && std::isfinite(d.x_max) && std::isfinite(d.z_min) &&
          std::isfinite(d.z_max)) || !(d.x_min < d.x_max) || !(d.z_min < d.z_max))
        return fail(SDD_E_ARG, "domain must be finite with x_min < x_max and z_min < z_max");
    if (m->n_materials < 1 || m->n_materials > SDD_MAX_MATERIALS)
        return fail(SDD_E_ARG, "n_materials must be in 1..8");
    if (m->n_eval < 1 || m->n_eval > SDD_MAX_EVAL) return fail(SDD_E_ARG, "n_eval must be in 1..32");
    if (!m->kappa) return fail(SDD_E_ARG, "kappa is NULL");
    for (int i = 0; i < m->n_eval * m->n_materials; ++i)
        if (!std::isfinite(m->kappa[i]) || m->kappa[i] < 0.0)
            return fail(SDD_E_ARG, "kappa must be finite and >= 0");
    const int K = m->n_materials;
    if (m->raster) {
        if (m->nx < 1 || m->nz < 1 || (long long)m->nx * m->nz > (1ll << 31))
            return fail(SDD_E_ARG, "raster size out of range");
        const long long n = (long long)m->nx * m->nz;
        for (long long i = 0; i < n; ++i)
            if (m->raster[i] < 0 || m->raster[i] >= K)
                return fail(SDD_E_ARG, "raster material id out of range");
    } else {
        if (m->bg_air < 0 || m->bg_air >= K || m->bg_earth < 0 || m->bg_earth >= K)
            return fail(SDD_E_ARG, "background material id out of range");
        if (m->n_shapes < 0 || m->n_shapes > SDD_MAX_SHAPES)
            return fail(SDD_E_ARG, "n_shapes must be in 0..16");
        if (m->n_shapes > 0 && !m->shapes) return fail(SDD_E_ARG, "shapes is NULL");
        for (int s = 0; s < m->n_shapes; ++s) {
            const sdd_shape &S = m->shapes[s];
            if (S.kind != SDD_SHAPE_RECT && S.kind != SDD_SHAPE_TRIANGLE)
                return fail(SDD_E_ARG, "unknown shape kind");
            if (S.material < 0 || S.material >= K) return fail(SDD_E_ARG, "shape material out of range");
            for (int j = 0; j < 6; ++j)
                if (std::isnan(S.v[j])) return fail(SDD_E_ARG, "shape coordinate is NaN");
        }
    }
    if (m->g_kind < SDD_G_COLUMNS || m->g_kind > SDD_G_X2MZ2) return fail(SDD_E_ARG, "unknown g_kind");
    if (m->g_kind == SDD_G_COLUMNS &&
        (m->g_left < 0 || m->g_left >= K || m->g_right < 0 || m->g_right >= K))
        return fail(SDD_E_ARG, "g_left / g_right out of range");
    return SDD_OK;
}

void build_model(const sdd_model_desc *m, ModelDev &M) {
    std::memset(&M, 0, sizeof(M));
    const sdd_domain &d = m->domain;
    M.xmin = d.x_min; M.xmax = d.x_max; M.zmin = d.z_min; M.zmax = d.z_max;
    M.xc = 0.5 * (d.x_min + d.x_max);
    M.zc = 0.5 * (d.z_min + d.z_max);
    M.hw = 0.5 * (d.x_max - d.x_min);
    M.hh = 0.5 * (d.z_max - d.z_min);
    M.K = m->n_materials;
    M.E = m->n_eval;
    int ep = 1;
    while (ep < M.E) ep <<= 1;
    M.Epad = ep;
    M.bg_air = m->bg_air;
    M.bg_earth = m->bg_earth;
    M.fhw = (float)M.hw; M.fhh = (float)M.hh;
    M.fxc = (float)M.xc; M.fzc = (float)M.zc;
    M.fzs = (float)(0.0 - M.zc);
    if (!m->raster) {
        M.n_shapes = m->n_shapes;
        for (int s = 0; s < m->n_shapes; ++s) {
            const sdd_shape &S = m->shapes[s];
            ShapeDev &D = M.shapes[s];
            D.kind = S.kind;
            D.mat = S.material;
            for (int j = 0; j < 6; ++j) D.d[j] = S.v[j];
            if (S.kind == SDD_SHAPE_RECT) {
                D.f[0] = (float)(S.v[0] - M.xc); D.f[1] = (float)(S.v[1] - M.xc);
                D.f[2] = (float)(S.v[2] - M.zc); D.f[3] = (float)(S.v[3] - M.zc);
                D.dsign = 1.0;
            } else {
                const double ax = S.v[0], az = S.v[1], bx = S.v[2], bz = S.v[3], cx = S.v[4], cz = S.v[5];
                const double area = (bx - ax) * (cz - az) - (bz - az) * (cx - ax);
                const double sg = area >= 0.0 ? 1.0 : -1.0;
                D.dsign = sg;
                // edge p->q: sg ((qx - px)(z - pz) - (qz - pz)(x - px)) >= 0, in centred coordinates
                const double px[3] = {ax, bx, cx}, pz[3] = {az, bz, cz};
                for (int e = 0; e < 3; ++e) {
                    const double x0 = px[e] - M.xc, z0 = pz[e] - M.zc;
                    const double x1 = px[(e + 1) % 3] - M.xc, z1 = pz[(e + 1) % 3] - M.zc;
                    const double A = -sg * (z1 - z0), B = sg * (x1 - x0);
                    const double C = -(A * x0 + B * z0);
                    D.f[3 * e + 0] = (float)A;
                    D.f[3 * e + 1] = (float)B;
                    D.f[3 * e + 2] = (float)C;
                }
            }
        }
        if (m->n_shapes == 0) M.gcode = GC_LAYER;
        else if (m->n_shapes == 1) M.gcode = m->shapes[0].kind == SDD_SHAPE_RECT ? GC_RECT1 : GC_TRI1;
        else if (m->n_shapes <= 4) M.gcode = GC_SHAPES4;
        else M.gcode = GC_SHAPES16;
        if (M.gcode == GC_RECT1) {
            // a vertical contact: the rectangle is the whole earth right of x0
            const sdd_shape &S = m->shapes[0];
            if (S.v[1] >= d.x_max && S.v[2] == 0.0 && S.v[3] >= d.z_max &&
                (float)(S.v[1] - M.xc) >= M.fhw && (float)(S.v[3] - M.zc) >= M.fhh)
                M.gcode = GC_CONTACT;
        }
    } else {
        M.gcode = GC_RASTER;
        M.nx = m->nx;
        M.nz = m->nz;
        M.sx = (double)m->nx / (d.x_max - d.x_min);
        M.sz = (double)m->nz / (d.z_max - d.z_min);
        M.fsx = (float)M.sx;
        M.fsz = (float)M.sz;
        M.fox = (float)(M.hw * M.sx - 0.5);
        M.foz = (float)(M.hh * M.sz - 0.5);
    }
    M.g_kind = m->g_kind;
    for (int j = 0; j < 6; ++j) M.g_coef[j] = m->g_coef[j];
    for (int i = 0; i < M.E * M.K; ++i) M.kappa[i] = m->kappa[i];
    for (int e = 0; e < M.E; ++e) {
        EvalDev &V = M.ev[e];
        if (m->g_kind != SDD_G_COLUMNS) continue;
        const double kl = m->kappa[e * M.K + m->g_left], kr = m->kappa[e * M.K + m->g_right];
        const std::complex<double> wl = std::sqrt(std::complex<double>(0.0, kl));
        const std::complex<double> wr = std::sqrt(std::complex<double>(0.0, kr));
        V.kl_re = wl.real(); V.kl_im = wl.imag();
        V.kr_re = wr.real(); V.kr_im = wr.imag();
        const auto tl = column_value(kl, d.z_min), tr = column_value(kr, d.z_min);
        const auto bl = column_value(kl, d.z_max), br = column_value(kr, d.z_max);
        V.tl_re = tl.real(); V.tl_im = tl.imag(); V.tr_re = tr.real(); V.tr_im = tr.imag();
        V.bl_re = bl.real(); V.bl_im = bl.imag(); V.br_re = br.real(); V.br_im = br.imag();
    }
}

// Fixed-order sum of the slots of each node's items (item order), then the
// mean and the standard errors of the real and imaginary parts.
__global__ void reduce_kernel(const double *__restrict__ slots, const int32_t *__restrict__ trunc,
                              const Item *__restrict__ items, const int32_t *__restrict__ node_item0,
                              int n_nodes, int E, double *__restrict__ mean, double *__restrict__ se) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_nodes * E) return;
    const int j = t / E, e = t % E;
    double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    long long nv = 0;
    for (int it = node_item0[j]; it < node_item0[j + 1]; ++it) {
        const double *o = slots + ((size_t)it * E + e) * 4;
        s0 += o[0]; s1 += o[1]; s2 += o[2]; s3 += o[3];
        nv += items[it].count - trunc[it];
    }
    const double N = (double)nv;
    double mr = nan(""), mi = nan(""), vr = nan(""), vi = nan("");
    if (nv > 0) { mr = s0 / N; mi = s1 / N; }
    if (nv > 1) {
        vr = fmax((s2 - s0 * mr) / (N - 1.0), 0.0);
        vi = fmax((s3 - s1 * mi) / (N - 1.0), 0.0);
    }
    mean[2 * t] = mr;
    mean[2 * t + 1] = mi;
    se[2 * t] = sqrt(vr / N);
    se[2 * t + 1] = sqrt(vi / N);
}

// Raw per-node sums (sum re, sum im, sum re^2, sum im^2 per evaluation, and the
// number of walks that reached the boundary), items of each node in order.
__global__ void sums_kernel(const double *__restrict__ slots, const int32_t *__restrict__ trunc,
                            const Item *__restrict__ items, const int32_t *__restrict__ node_item0,
                            int n_nodes, int E, double *__restrict__ sums, long long *__restrict__ nvalid) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_nodes * E) return;
    const int j = t / E, e = t % E;
    double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    long long nv = 0;
    for (int it = node_item0[j]; it < node_item0[j + 1]; ++it) {
        const double *o = slots + ((size_t)it * E + e) * 4;
        s0 += o[0]; s1 += o[1]; s2 += o[2]; s3 += o[3];
        nv += items[it].count - trunc[it];
    }
    sums[4 * t + 0] = s0;
    sums[4 * t + 1] = s1;
    sums[4 * t + 2] = s2;
    sums[4 * t + 3] = s3;
    if (e == 0) nvalid[j] = nv;
}

struct Plan {
    std::vector<Item> items;
    std::vector<int32_t> node_item0;  // [n_nodes + 1]
    long long total_paths = 0;
    bool cached = false;     // identical to the table already on the device
    bool cacheable = false;  // may be reused by a later call with the same key
};

sdd_status check_call(sdd_ctx *ctx, int32_t n_nodes, const int64_t *n_paths, double dt,
                      const sdd_config *cfg) {
    if (!ctx) return fail(SDD_E_ARG, "ctx is NULL");
    if (n_nodes < 0) return fail(SDD_E_ARG, "n_nodes < 0");
    if (n_nodes > 0 && !n_paths) return fail(SDD_E_ARG, "n_paths is NULL");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(SDD_E_ARG, "dt must be finite and > 0");
    for (int j = 0; j < n_nodes; ++j)
        if (n_paths[j] < 1 || n_paths[j] > 0x7fffffffll)
            return fail(SDD_E_ARG, "n_paths must be in 1..2^31-1");
    if (cfg) {
        if (cfg->precision != SDD_FP32 && cfg->precision != SDD_FP64)
            return fail(SDD_E_ARG, "precision must be SDD_FP32 or SDD_FP64");
        if (cfg->max_steps < 0 || cfg->max_steps > kMaxSteps)
            return fail(SDD_E_ARG, "max_steps must be in 0..2^26");
        if (cfg->block_threads != 0 &&
            (cfg->block_threads % 32 != 0 || cfg->block_threads < 32 || cfg->block_threads > 256))
            return fail(SDD_E_ARG, "block_threads must be a multiple of 32 in 32..256");
        if (cfg->ctas_per_sm < 0 || cfg->chunk_paths < 0)
            return fail(SDD_E_ARG, "ctas_per_sm and chunk_paths must be >= 0");
    }
    return SDD_OK;
}

sdd_status check_nodes(const sdd_ctx *ctx, const double *xz, int32_t n) {
    for (int j = 0; j < n; ++j) {
        const double x = xz[2 * j], z = xz[2 * j + 1];
        if (!(x > ctx->M.xmin && x < ctx->M.xmax && z > ctx->M.zmin && z < ctx->M.zmax))
            return fail(SDD_E_ARG, "node " + std::to_string(j) + " is not strictly inside the domain");
    }
    return SDD_OK;
}

struct Launch {
    bool f64;
    int kmax, block, grid, chunk;
    int64_t max_steps;
};

Launch choose_launch(const sdd_ctx *ctx, const sdd_config *cfg, double dt, long long total_paths) {
    Launch L;
    L.f64 = cfg && cfg->precision == SDD_FP64;
    L.kmax = kmax_for(ctx->K);
    L.block = (cfg && cfg->block_threads) ? cfg->block_threads : 256;
    int occ = L.f64 ? occupancy_f64(L.kmax, ctx->geo, L.block)
                    : occupancy_f32(L.kmax, ctx->M.gcode, L.block);
    if (occ < 1) occ = 1;
    if (cfg && cfg->ctas_per_sm > 0 && cfg->ctas_per_sm < occ) occ = cfg->ctas_per_sm;
    L.grid = ctx->n_sm * occ;
    const long long warps = (long long)L.grid * (L.block / 32);
    long long chunk = (cfg && cfg->chunk_paths) ? cfg->chunk_paths : 0;
    if (chunk == 0) {
        chunk = (total_paths + warps * 6 - 1) / (warps * 6);
        chunk = (chunk + 31) / 32 * 32;
        if (chunk < 32) chunk = 32;
        if (chunk > 16384) chunk = 16384;
    }
    L.chunk = (int)chunk;
    L.max_steps = (cfg && cfg->max_steps) ? cfg->max_steps : (int64_t)std::ceil(20.0 / dt);
    if (L.max_steps > kMaxSteps) L.max_steps = kMaxSteps;
    L.max_steps += L.max_steps & 1;  // walks advance two steps per random-number call
    return L;
}

Plan plan_items(int32_t n_nodes, const int64_t *n_paths, int chunk, uint32_t p_offset) {
    Plan P;
    P.node_item0.resize(n_nodes + 1);
    for (int j = 0; j < n_nodes; ++j) {
        P.node_item0[j] = (int32_t)P.items.size();
        for (int64_t p = 0; p < n_paths[j]; p += chunk) {
            Item I;
            I.node = j;
            I.path0 = p_offset + (uint32_t)p;
            I.count = (int32_t)std::min<int64_t>(chunk, n_paths[j] - p);
            I.pad = 0;
            P.items.push_back(I);
        }
        P.total_paths += n_paths[j];
    }
    P.node_item0[n_nodes] = (int32_t)P.items.size();
    return P;
}

// Plan the items of a call; reuse the device copy of the previous table when
// the call has the same path counts, chunk and path offset.
Plan plan_cached(sdd_ctx *ctx, int32_t n_nodes, const int64_t *n_paths, int chunk,
                 uint32_t p_offset, bool cacheable) {
    Plan P = plan_items(n_nodes, n_paths, chunk, p_offset);
    const bool same = cacheable && ctx->plan_valid && ctx->plan_chunk == chunk &&
                      ctx->plan_offset == p_offset && (int32_t)ctx->plan_paths.size() == n_nodes &&
                      std::equal(ctx->plan_paths.begin(), ctx->plan_paths.end(), n_paths);
    P.cached = same;
    P.cacheable = cacheable;
    if (!same) {
        // the device table becomes valid for this key only once its upload is queued
        ctx->plan_valid = false;
        if (cacheable) {
            ctx->plan_paths.assign(n_paths, n_paths + n_nodes);
            ctx->plan_chunk = chunk;
            ctx->plan_offset = p_offset;
        }
    }
    return P;
}

// Items for paths [begin[j], begin[j] + count[j]) of every node.
Plan plan_ranges(int32_t n_nodes, const int64_t *begin, const int64_t *count, int chunk) {
    Plan P;
    P.node_item0.resize(n_nodes + 1);
    for (int j = 0; j < n_nodes; ++j) {
        P.node_item0[j] = (int32_t)P.items.size();
        for (int64_t p = 0; p < count[j]; p += chunk) {
            Item I;
            I.node = j;
            I.path0 = (uint32_t)(begin[j] + p);
            I.count = (int32_t)std::min<int64_t>(chunk, count[j] - p);
            I.pad = 0;
            P.items.push_back(I);
        }
        P.total_paths += count[j];
    }
    P.node_item0[n_nodes] = (int32_t)P.items.size();
    return P;
}

WalkArgs base_args(sdd_ctx *ctx, const Launch &L, double dt, uint64_t seed) {
    WalkArgs A;
    std::memset(&A, 0, sizeof(A));
    A.dt = dt;
    A.sdt = std::sqrt(dt);
    A.f_cdt = (float)(-2.0 * std::log(2.0) * dt);
    A.f_c2dt = (float)(2.0 / dt);
    // single-precision bridge uniforms are >= 2^-19, so a hit needs
    // 2 d d' / dt <= -ln U <= 19 ln 2; 1e-3 margin for rounding
    A.f_bthr = (float)(19.0 * std::log(2.0) * dt / 2.0 * 1.001);
    A.key0 = (uint32_t)(seed & 0xffffffffu);
    A.key1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        A.rk0[r] = A.key0 + (uint32_t)r * 0x9E3779B9u;
        A.rk1[r] = A.key1 + (uint32_t)r * 0xBB67AE85u;
    }
    A.max_steps = (uint32_t)L.max_steps;
    return A;
}

// Upload the item table (through pinned staging) and launch walk + reduce.
sdd_status run(sdd_ctx *ctx, const Plan &P, const Launch &L, WalkArgs A, cudaStream_t s,
               bool timed, bool do_reduce, double *d_mean, double *d_se, int n_nodes) {
    const size_t ni = P.items.size();
    if (ni == 0) return SDD_OK;
    SDD_CUDA(ctx->items.ensure(ni * sizeof(Item) + (n_nodes + 1) * sizeof(int32_t)));
    SDD_CUDA(ctx->slots.ensure(ni * (size_t)ctx->E * 4 * sizeof(double)));
    SDD_CUDA(ctx->trunc.ensure(ni * sizeof(int32_t)));
    SDD_CUDA(ctx->counters.ensure(3 * sizeof(unsigned long long)));
    SDD_CUDA(ctx->queue.ensure(sizeof(int32_t)));
    SDD_CUDA(ctx->err.ensure(sizeof(int32_t)));
    const size_t hbytes = ni * sizeof(Item) + (n_nodes + 1) * sizeof(int32_t);
    ctx->last_h2d = 0;
    if (!P.cached) {
        if (ctx->items_done) SDD_CUDA(cudaEventSynchronize(ctx->items_done));
        if (hbytes > ctx->h_items_cap) {
            if (ctx->h_items) cudaFreeHost(ctx->h_items);
            ctx->h_items = nullptr;
            ctx->h_items_cap = 0;
            SDD_CUDA(cudaMallocHost((void **)&ctx->h_items, hbytes + hbytes / 4 + 256));
            ctx->h_items_cap = hbytes + hbytes / 4 + 256;
        }
        std::memcpy(ctx->h_items, P.items.data(), ni * sizeof(Item));
        std::memcpy(reinterpret_cast<unsigned char *>(ctx->h_items) + ni * sizeof(Item),
                    P.node_item0.data(), (n_nodes + 1) * sizeof(int32_t));
        SDD_CUDA(cudaMemcpyAsync(ctx->items.p, ctx->h_items, hbytes, cudaMemcpyHostToDevice, s));
        SDD_CUDA(cudaEventRecord(ctx->items_done, s));
        ctx->last_h2d = hbytes;
        ctx->plan_valid = P.cacheable;
    }
    SDD_CUDA(cudaMemsetAsync(ctx->queue.p, 0, sizeof(int32_t), s));
    SDD_CUDA(cudaMemsetAsync(ctx->counters.p, 0, 3 * sizeof(unsigned long long), s));
    A.items = (const Item *)ctx->items.p;
    A.n_items = (int32_t)ni;
    A.slots = (double *)ctx->slots.p;
    A.item_trunc = (int32_t *)ctx->trunc.p;
    A.counters = (unsigned long long *)ctx->counters.p;
    A.queue = (int32_t *)ctx->queue.p;
    A.error = (int32_t *)ctx->err.p;
    const int warps_per_cta = L.block / 32;
    int grid = L.grid;
    const int need = (int)((ni + warps_per_cta - 1) / warps_per_cta);
    if (grid > need) grid = need;
    if (timed) SDD_CUDA(cudaEventRecord(ctx->ev0, s));
    cudaError_t e = L.f64 ? launch_walk_f64(L.kmax, ctx->geo, ctx->M, A, grid, L.block, s)
                          : launch_walk_f32(L.kmax, ctx->geo, ctx->M, A, grid, L.block, s);
    if (e != cudaSuccess) return cuda_fail(e, "walk kernel launch");
    if (timed) SDD_CUDA(cudaEventRecord(ctx->ev1, s));
    if (do_reduce) {
        const int nt = n_nodes * ctx->E;
        const Item *d_items = (const Item *)ctx->items.p;
        const int32_t *d_i0 = (const int32_t *)(reinterpret_cast<unsigned char *>(ctx->items.p) + ni * sizeof(Item));
        reduce_kernel<<<(nt + 127) / 128, 128, 0, s>>>((const double *)ctx->slots.p,
                                                      (const int32_t *)ctx->trunc.p, d_items, d_i0,
                                                      n_nodes, ctx->E, d_mean, d_se);
        SDD_CUDA(cudaGetLastError());
    }
    return SDD_OK;
}

}  // namespace

extern "C" {

const char *sdd_status_str(sdd_status s) {
    switch (s) {
    case SDD_OK: return "ok";
    case SDD_E_ARG: return "invalid argument";
    case SDD_E_OOM: return "out of memory";
    case SDD_E_CUDA: return "CUDA error";
    case SDD_E_TRUNCATED: return "some walks reached max_steps (results valid)";
    case SDD_E_CANCELLED: return "cancelled";
    case SDD_E_TIMEOUT: return "timed out";
    case SDD_E_UNSUPPORTED: return "unsupported configuration";
    case SDD_E_BUSY: return "busy: no free slot or memory";
    }
    return "unknown status";
}

const char *sdd_last_error(void) { return g_last_error.c_str(); }

sdd_status sdd_create(const sdd_model_desc *model, sdd_ctx **out) {
    if (!out) return fail(SDD_E_ARG, "out is NULL");
    *out = nullptr;
    sdd_status st = check_model(model);
    if (st != SDD_OK) return st;
    sdd_ctx *c = new (std::nothrow) sdd_ctx();
    if (!c) return fail(SDD_E_OOM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev1);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->items_done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        sdd_destroy(c);
        return cuda_fail(e, "context setup");
    }
    build_model(model, c->M);
    c->K = model->n_materials;
    c->E = model->n_eval;
    if (model->raster) {
        c->geo = GEO_RASTER;
        const size_t nb = (size_t)model->nx * model->nz;
        e = c->raster.ensure(nb);
        if (e == cudaSuccess) e = cudaMemcpy(c->raster.p, model->raster, nb, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            sdd_destroy(c);
            return e == cudaErrorMemoryAllocation ? fail(SDD_E_OOM, "raster allocation")
                                                  : cuda_fail(e, "raster upload");
        }
        c->M.raster = (const int8_t *)c->raster.p;
    }
    *out = c;
    return SDD_OK;
}

void sdd_destroy(sdd_ctx *c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    DevBuf *bufs[] = {&c->raster, &c->items, &c->slots, &c->trunc, &c->counters, &c->queue,
                      &c->err, &c->nodes, &c->node_ids, &c->mean, &c->se, &c->rec_steps,
                      &c->rec_counts, &c->rec_exit, &c->rec_wall, &c->rec_mlast};
    for (DevBuf *b : bufs) b->release();
    if (c->h_items) cudaFreeHost(c->h_items);
    if (c->items_done) cudaEventDestroy(c->items_done);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

int32_t sdd_n_eval(const sdd_ctx *c) { return c ? c->E : 0; }
int32_t sdd_n_materials(const sdd_ctx *c) { return c ? c->K : 0; }

sdd_status sdd_interface_values(sdd_ctx *ctx, const double *nodes_xz, const uint32_t *node_ids,
                                int32_t n_nodes, const int64_t *n_paths, double dt,
                                uint64_t seed, const sdd_config *cfg, double *mean, double *se,
                                sdd_stats *stats) {
    sdd_status st = check_call(ctx, n_nodes, n_paths, dt, cfg);
    if (st != SDD_OK) return st;
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (n_nodes == 0) return SDD_OK;
    if (!nodes_xz || !mean || !se) return fail(SDD_E_ARG, "nodes_xz, mean and se must not be NULL");
    st = check_nodes(ctx, nodes_xz, n_nodes);
    if (st != SDD_OK) return st;
    long long total = 0;
    for (int j = 0; j < n_nodes; ++j) total += n_paths[j];
    const Launch L = choose_launch(ctx, cfg, dt, total);
    const Plan P = plan_cached(ctx, n_nodes, n_paths, L.chunk, 0, true);
    cudaStream_t s = ctx->stream;
    const size_t ob = (size_t)n_nodes * ctx->E * 2 * sizeof(double);
    SDD_CUDA(ctx->nodes.ensure((size_t)n_nodes * 2 * sizeof(double)));
    SDD_CUDA(ctx->mean.ensure(ob));
    SDD_CUDA(ctx->se.ensure(ob));
    SDD_CUDA(cudaMemcpyAsync(ctx->nodes.p, nodes_xz, (size_t)n_nodes * 2 * sizeof(double),
                             cudaMemcpyHostToDevice, s));
    WalkArgs A = base_args(ctx, L, dt, seed);
    A.nodes = (const double *)ctx->nodes.p;
    if (node_ids) {
        SDD_CUDA(ctx->node_ids.ensure((size_t)n_nodes * sizeof(uint32_t)));
        SDD_CUDA(cudaMemcpyAsync(ctx->node_ids.p, node_ids, (size_t)n_nodes * sizeof(uint32_t),
                                 cudaMemcpyHostToDevice, s));
        A.node_ids = (const uint32_t *)ctx->node_ids.p;
    }
    st = run(ctx, P, L, A, s, true, true, (double *)ctx->mean.p, (double *)ctx->se.p, n_nodes);
    if (st != SDD_OK) return st;
    unsigned long long cnt[3] = {0, 0, 0};
    SDD_CUDA(cudaMemcpyAsync(mean, ctx->mean.p, ob, cudaMemcpyDeviceToHost, s));
    SDD_CUDA(cudaMemcpyAsync(se, ctx->se.p, ob, cudaMemcpyDeviceToHost, s));
    SDD_CUDA(cudaMemcpyAsync(cnt, ctx->counters.p, sizeof(cnt), cudaMemcpyDeviceToHost, s));
    SDD_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    SDD_CUDA(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
    if (stats) {
        stats->h2d_bytes = ctx->last_h2d + (uint64_t)n_nodes * 2 * sizeof(double) +
                           (node_ids ? (uint64_t)n_nodes * sizeof(uint32_t) : 0);
        stats->d2h_bytes = 2 * ob + sizeof(cnt);
        stats->steps = cnt[0];
        stats->walks = cnt[1];
        stats->truncated = cnt[2];
        stats->kernel_ms = ms;
        stats->launches = 2;
        stats->items = (int32_t)P.items.size();
        stats->grid = L.grid;
        stats->block = L.block;
    }
    return cnt[2] ? SDD_E_TRUNCATED : SDD_OK;
}

sdd_status sdd_interface_values_device(sdd_ctx *ctx, const double *d_nodes_xz,
                                       const uint32_t *d_node_ids, int32_t n_nodes,
                                       const int64_t *n_paths, double dt, uint64_t seed,
                                       const sdd_config *cfg, double *d_mean, double *d_se,
                                       uint64_t *d_counters, void *stream) {
    sdd_status st = check_call(ctx, n_nodes, n_paths, dt, cfg);
    if (st != SDD_OK) return st;
    if (n_nodes == 0) return SDD_OK;
    if (!d_nodes_xz || !d_mean || !d_se) return fail(SDD_E_ARG, "d_nodes_xz, d_mean and d_se must not be NULL");
    long long total = 0;
    for (int j = 0; j < n_nodes; ++j) total += n_paths[j];
    const Launch L = choose_launch(ctx, cfg, dt, total);
    const Plan P = plan_cached(ctx, n_nodes, n_paths, L.chunk, 0, true);
    cudaStream_t s = (cudaStream_t)stream;
    WalkArgs A = base_args(ctx, L, dt, seed);
    A.nodes = d_nodes_xz;
    A.node_ids = d_node_ids;
    st = run(ctx, P, L, A, s, false, true, d_mean, d_se, n_nodes);
    if (st != SDD_OK) return st;
    if (d_counters)
        SDD_CUDA(cudaMemcpyAsync(d_counters, ctx->counters.p, 3 * sizeof(uint64_t),
                                 cudaMemcpyDeviceToDevice, s));
    return SDD_OK;
}

sdd_status sdd_walk_records(sdd_ctx *ctx, double x0, double z0, uint32_t node_id, uint32_t p0,
                            int32_t count, double dt, uint64_t seed, const sdd_config *cfg,
                            int64_t *steps, int64_t *counts, double *exit_xzt, int32_t *wall,
                            int32_t *m_last) {
    const int64_t np = count;
    sdd_status st = check_call(ctx, count > 0 ? 1 : 0, &np, dt, cfg);
    if (st != SDD_OK) return st;
    if (count <= 0) return count == 0 ? SDD_OK : fail(SDD_E_ARG, "count < 0");
    if (!steps) return fail(SDD_E_ARG, "steps must not be NULL");
    if ((uint64_t)p0 + (uint64_t)count > 0x100000000ull) return fail(SDD_E_ARG, "path range overflows 32 bits");
    const double xz[2] = {x0, z0};
    st = check_nodes(ctx, xz, 1);
    if (st != SDD_OK) return st;
    const Launch L = choose_launch(ctx, cfg, dt, count);
    const Plan P = plan_cached(ctx, 1, &np, L.chunk, p0, false);
    cudaStream_t s = ctx->stream;
    SDD_CUDA(ctx->nodes.ensure(2 * sizeof(double)));
    SDD_CUDA(ctx->node_ids.ensure(sizeof(uint32_t)));
    SDD_CUDA(ctx->rec_steps.ensure((size_t)count * 8));
    SDD_CUDA(ctx->rec_counts.ensure((size_t)count * ctx->K * 8));
    SDD_CUDA(ctx->rec_exit.ensure((size_t)count * 3 * 8));
    SDD_CUDA(ctx->rec_wall.ensure((size_t)count * 4));
    SDD_CUDA(ctx->rec_mlast.ensure((size_t)count * 4));
    SDD_CUDA(cudaMemcpyAsync(ctx->nodes.p, xz, sizeof(xz), cudaMemcpyHostToDevice, s));
    SDD_CUDA(cudaMemcpyAsync(ctx->node_ids.p, &node_id, sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    WalkArgs A = base_args(ctx, L, dt, seed);
    A.nodes = (const double *)ctx->nodes.p;
    A.node_ids = (const uint32_t *)ctx->node_ids.p;
    A.rec_steps = (int64_t *)ctx->rec_steps.p;
    A.rec_counts = (int64_t *)ctx->rec_counts.p;
    A.rec_exit = (double *)ctx->rec_exit.p;
    A.rec_wall = (int32_t *)ctx->rec_wall.p;
    A.rec_mlast = (int32_t *)ctx->rec_mlast.p;
    st = run(ctx, P, L, A, s, false, false, nullptr, nullptr, 1);
    if (st != SDD_OK) return st;
    SDD_CUDA(cudaMemcpyAsync(steps, ctx->rec_steps.p, (size_t)count * 8, cudaMemcpyDeviceToHost, s));
    if (counts)
        SDD_CUDA(cudaMemcpyAsync(counts, ctx->rec_counts.p, (size_t)count * ctx->K * 8, cudaMemcpyDeviceToHost, s));
    if (exit_xzt)
        SDD_CUDA(cudaMemcpyAsync(exit_xzt, ctx->rec_exit.p, (size_t)count * 24, cudaMemcpyDeviceToHost, s));
    if (wall) SDD_CUDA(cudaMemcpyAsync(wall, ctx->rec_wall.p, (size_t)count * 4, cudaMemcpyDeviceToHost, s));
    if (m_last) SDD_CUDA(cudaMemcpyAsync(m_last, ctx->rec_mlast.p, (size_t)count * 4, cudaMemcpyDeviceToHost, s));
    SDD_CUDA(cudaStreamSynchronize(s));
    return SDD_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Entry point that allocates nothing (sdd_interface_values_noalloc).
//
// Some callers cannot call cudaMalloc: hosts that hand out all device memory
// from their own fixed arena, processes whose device memory is already
// reserved by another framework's caching allocator, and latency-critical
// loops that cannot afford the device-wide synchronisation cudaMalloc and
// cudaFree may imply.  For them the per-call scratch of the walk -- work-item
// table, per-item partial sums, counters -- lives in this file-scope device
// array, which every GPU that loads the library holds until the process
// exits.  Every call shares it, so calls that overlap on the GPU (on
// different streams, or from different host threads) race; the array keeps
// the last call's contents and each call clears what must start at zero.

namespace {

constexpr size_t kNaItems = SDD_NOALLOC_MAX_ITEMS;
constexpr size_t kNaNodes = SDD_NOALLOC_MAX_NODES;
// layout (bytes, each part 256-aligned)
constexpr size_t kNaOffItems = 0;
constexpr size_t kNaOffNodeItem0 = kNaOffItems + kNaItems * sizeof(Item);
constexpr size_t kNaOffPaths = kNaOffNodeItem0 + ((kNaNodes + 1) * 4 + 255) / 256 * 256;
constexpr size_t kNaOffTrunc = kNaOffPaths + kNaNodes * 8;
constexpr size_t kNaOffCount = kNaOffTrunc + kNaItems * 4;
constexpr size_t kNaOffSlots = kNaOffCount + 256;  // counters (3 x u64), queue, error
constexpr size_t kNaBytes = kNaOffSlots + kNaItems * (size_t)kMaxE * 4 * sizeof(double);
static_assert(kNaBytes == SDD_NOALLOC_SCRATCH_BYTES, "scratch size differs from sdd.h");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

// Device address of g_noalloc_scratch per device, looked up once per device
// with that device current (the name is only a host-side stand-in).
constexpr int kNaMaxDevices = 64;
unsigned char *g_noalloc_ptr[kNaMaxDevices] = {nullptr};

sdd_status noalloc_scratch(int device, unsigned char **out) {
    if (device < 0 || device >= kNaMaxDevices) return fail(SDD_E_UNSUPPORTED, "device id too large");
    if (!g_noalloc_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_noalloc_ptr[device] = static_cast<unsigned char *>(p);
    }
    *out = g_noalloc_ptr[device];
    return SDD_OK;
}

// Work-item table of the no-allocation call, built on the device from the
// per-node path counts in the scratch array (one CTA).
__global__ void noalloc_plan_kernel(int n_nodes, int chunk) {
    Item *items = reinterpret_cast<Item *>(g_noalloc_scratch + kNaOffItems);
    int32_t *node_item0 = reinterpret_cast<int32_t *>(g_noalloc_scratch + kNaOffNodeItem0);
    const int64_t *n_paths = reinterpret_cast<const int64_t *>(g_noalloc_scratch + kNaOffPaths);
    if (threadIdx.x == 0) {
        int32_t acc = 0;
        for (int j = 0; j < n_nodes; ++j) {
            node_item0[j] = acc;
            acc += (int32_t)((n_paths[j] + chunk - 1) / chunk);
        }
        node_item0[n_nodes] = acc;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < n_nodes; j += blockDim.x) {
        int32_t it = node_item0[j];
        for (int64_t p = 0; p < n_paths[j]; p += chunk, ++it) {
            Item I;
            I.node = j;
            I.path0 = (uint32_t)p;
            I.count = (int32_t)(n_paths[j] - p < chunk ? n_paths[j] - p : chunk);
            I.pad = 0;
            items[it] = I;
        }
    }
}

}  // namespace

extern "C" sdd_status sdd_interface_values_noalloc(sdd_ctx *ctx, const double *d_nodes_xz,
                                                   const uint32_t *d_node_ids, int32_t n_nodes,
                                                   const int64_t *n_paths, double dt,
                                                   uint64_t seed, const sdd_config *cfg,
                                                   double *d_mean, double *d_se,
                                                   uint64_t *d_counters, void *stream) {
    sdd_status st = check_call(ctx, n_nodes, n_paths, dt, cfg);
    if (st != SDD_OK) return st;
    if (n_nodes == 0) return SDD_OK;
    if (!d_nodes_xz || !d_mean || !d_se) return fail(SDD_E_ARG, "d_nodes_xz, d_mean and d_se must not be NULL");
    if ((size_t)n_nodes > kNaNodes)
        return fail(SDD_E_ARG, "sdd_interface_values_noalloc takes at most SDD_NOALLOC_MAX_NODES (" +
                                   std::to_string(kNaNodes) + ") nodes per call");
    int device = -1;
    SDD_CUDA(cudaGetDevice(&device));
    if (device != ctx->device) return fail(SDD_E_ARG, "the context's device is not the current device");
    unsigned char *base = nullptr;
    st = noalloc_scratch(device, &base);
    if (st != SDD_OK) return st;

    long long total = 0;
    for (int j = 0; j < n_nodes; ++j) total += n_paths[j];
    Launch L = choose_launch(ctx, cfg, dt, total);
    // widen the chunks until the work items fit the scratch array
    long long chunk = L.chunk;
    const long long room = (long long)kNaItems - n_nodes;
    if (chunk * room < total) chunk = (total + room - 1) / room;
    long long n_items = 0;
    for (int j = 0; j < n_nodes; ++j) n_items += (n_paths[j] + chunk - 1) / chunk;
    if (n_items > (long long)kNaItems || chunk > 0x7fffffffll)
        return fail(SDD_E_ARG, "request does not fit the no-allocation scratch limits");
    L.chunk = (int)chunk;

    cudaStream_t s = (cudaStream_t)stream;
    SDD_CUDA(cudaMemcpyAsync(base + kNaOffPaths, n_paths, (size_t)n_nodes * sizeof(int64_t),
                             cudaMemcpyHostToDevice, s));
    SDD_CUDA(cudaMemsetAsync(base + kNaOffCount, 0, 256, s));
    noalloc_plan_kernel<<<1, 256, 0, s>>>(n_nodes, L.chunk);
    SDD_CUDA(cudaGetLastError());

    WalkArgs A = base_args(ctx, L, dt, seed);
    A.nodes = d_nodes_xz;
    A.node_ids = d_node_ids;
    A.items = reinterpret_cast<const Item *>(base + kNaOffItems);
    A.n_items = (int32_t)n_items;
    A.slots = reinterpret_cast<double *>(base + kNaOffSlots);
    A.item_trunc = reinterpret_cast<int32_t *>(base + kNaOffTrunc);
    A.counters = reinterpret_cast<unsigned long long *>(base + kNaOffCount);
    A.queue = reinterpret_cast<int32_t *>(base + kNaOffCount + 3 * sizeof(unsigned long long));
    A.error = A.queue + 1;
    const int warps_per_cta = L.block / 32;
    int grid = L.grid;
    const int need = (int)((n_items + warps_per_cta - 1) / warps_per_cta);
    if (grid > need) grid = need;
    cudaError_t e = L.f64 ? launch_walk_f64(L.kmax, ctx->geo, ctx->M, A, grid, L.block, s)
                          : launch_walk_f32(L.kmax, ctx->geo, ctx->M, A, grid, L.block, s);
    if (e != cudaSuccess) return cuda_fail(e, "walk kernel launch");
    const int nt = n_nodes * ctx->E;
    reduce_kernel<<<(nt + 127) / 128, 128, 0, s>>>(
        A.slots, A.item_trunc, A.items, reinterpret_cast<const int32_t *>(base + kNaOffNodeItem0),
        n_nodes, ctx->E, d_mean, d_se);
    SDD_CUDA(cudaGetLastError());
    if (d_counters)
        SDD_CUDA(cudaMemcpyAsync(d_counters, A.counters, 3 * sizeof(uint64_t),
                                 cudaMemcpyDeviceToDevice, s));
    return SDD_OK;
}

// ---------------------------------------------------------------------------
// Adaptive path counts (sdd_interface_values_target).

namespace {

// Walks of one phase, and the raw per-node sums of the phase on the host.
sdd_status run_phase(sdd_ctx *ctx, const Plan &P, const Launch &L, const WalkArgs &A0,
                     int32_t n_nodes, std::vector<double> &sums, std::vector<long long> &nvalid,
                     unsigned long long cnt[3], float *ms) {
    sums.assign((size_t)n_nodes * ctx->E * 4, 0.0);
    nvalid.assign(n_nodes, 0);
    cnt[0] = cnt[1] = cnt[2] = 0;
    *ms = 0.f;
    if (P.items.empty()) return SDD_OK;
    cudaStream_t s = ctx->stream;
    sdd_status st = run(ctx, P, L, A0, s, true, false, nullptr, nullptr, n_nodes);
    if (st != SDD_OK) return st;
    const size_t ni = P.items.size();
    SDD_CUDA(ctx->mean.ensure(sums.size() * sizeof(double)));
    SDD_CUDA(ctx->se.ensure((size_t)n_nodes * sizeof(long long)));
    const Item *d_items = (const Item *)ctx->items.p;
    const int32_t *d_i0 = (const int32_t *)(reinterpret_cast<unsigned char *>(ctx->items.p) + ni * sizeof(Item));
    const int nt = n_nodes * ctx->E;
    sums_kernel<<<(nt + 127) / 128, 128, 0, s>>>((const double *)ctx->slots.p, (const int32_t *)ctx->trunc.p,
                                                d_items, d_i0, n_nodes, ctx->E, (double *)ctx->mean.p,
                                                (long long *)ctx->se.p);
    SDD_CUDA(cudaGetLastError());
    SDD_CUDA(cudaMemcpyAsync(sums.data(), ctx->mean.p, sums.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    SDD_CUDA(cudaMemcpyAsync(nvalid.data(), ctx->se.p, (size_t)n_nodes * sizeof(long long), cudaMemcpyDeviceToHost, s));
    SDD_CUDA(cudaMemcpyAsync(cnt, ctx->counters.p, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    SDD_CUDA(cudaStreamSynchronize(s));
    SDD_CUDA(cudaEventElapsedTime(ms, ctx->ev0, ctx->ev1));
    return SDD_OK;
}

// mean and standard error of each component from the raw sums
void finish(const double *q, long long nv, double *mean, double *se) {
    const double N = (double)nv;
    double mr = nan(""), mi = nan(""), vr = nan(""), vi = nan("");
    if (nv > 0) { mr = q[0] / N; mi = q[1] / N; }
    if (nv > 1) {
        vr = std::max((q[2] - q[0] * mr) / (N - 1.0), 0.0);
        vi = std::max((q[3] - q[1] * mi) / (N - 1.0), 0.0);
    }
    mean[0] = mr; mean[1] = mi;
    se[0] = std::sqrt(vr / N); se[1] = std::sqrt(vi / N);
}

}  // namespace

extern "C" sdd_status sdd_interface_values_target(sdd_ctx *ctx, const double *nodes_xz,
                                                  const uint32_t *node_ids, int32_t n_nodes,
                                                  int64_t n_pilot, int64_t n_max, double target_se,
                                                  double dt, uint64_t seed, const sdd_config *cfg,
                                                  double *mean, double *se, int64_t *n_used,
                                                  sdd_stats *stats) {
    if (!(target_se > 0.0) || !std::isfinite(target_se)) return fail(SDD_E_ARG, "target_se must be finite and > 0");
    if (n_pilot < 2 || n_max < n_pilot || n_max > 0x7fffffffll)
        return fail(SDD_E_ARG, "need 2 <= n_pilot <= n_max <= 2^31-1");
    std::vector<int64_t> pilot((size_t)std::max(n_nodes, 0), n_pilot);
    sdd_status st = check_call(ctx, n_nodes, pilot.data(), dt, cfg);
    if (st != SDD_OK) return st;
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (n_nodes == 0) return SDD_OK;
    if (!nodes_xz || !mean || !se) return fail(SDD_E_ARG, "nodes_xz, mean and se must not be NULL");
    st = check_nodes(ctx, nodes_xz, n_nodes);
    if (st != SDD_OK) return st;
    cudaStream_t s = ctx->stream;
    SDD_CUDA(ctx->nodes.ensure((size_t)n_nodes * 2 * sizeof(double)));
    SDD_CUDA(cudaMemcpyAsync(ctx->nodes.p, nodes_xz, (size_t)n_nodes * 2 * sizeof(double),
                             cudaMemcpyHostToDevice, s));
    const int E = ctx->E;
    std::vector<int64_t> begin((size_t)n_nodes, 0), extra((size_t)n_nodes, 0);

    // phase 1: the pilot walks of every node
    Launch L = choose_launch(ctx, cfg, dt, (long long)n_pilot * n_nodes);
    WalkArgs A = base_args(ctx, L, dt, seed);
    A.nodes = (const double *)ctx->nodes.p;
    if (node_ids) {
        SDD_CUDA(ctx->node_ids.ensure((size_t)n_nodes * sizeof(uint32_t)));
        SDD_CUDA(cudaMemcpyAsync(ctx->node_ids.p, node_ids, (size_t)n_nodes * sizeof(uint32_t),
                                 cudaMemcpyHostToDevice, s));
        A.node_ids = (const uint32_t *)ctx->node_ids.p;
    }
    ctx->plan_valid = false;
    Plan P1 = plan_ranges(n_nodes, begin.data(), pilot.data(), L.chunk);
    std::vector<double> s1, s2;
    std::vector<long long> v1, v2;
    unsigned long long c1[3], c2[3];
    float ms1 = 0.f, ms2 = 0.f;
    st = run_phase(ctx, P1, L, A, n_nodes, s1, v1, c1, &ms1);
    if (st != SDD_OK) return st;

    // path count each node needs: N = clamp(ceil(max_e (var_re + var_im) / se^2), n_pilot, n_max)
    long long total2 = 0;
    for (int j = 0; j < n_nodes; ++j) {
        double need = 0.0;
        for (int e = 0; e < E; ++e) {
            double m[2], sd[2];
            finish(&s1[((size_t)j * E + e) * 4], v1[j], m, sd);
            const double var = (sd[0] * sd[0] + sd[1] * sd[1]) * (double)v1[j];
            if (std::isfinite(var)) need = std::max(need, var);
        }
        double N = std::ceil(need / (target_se * target_se));
        if (!(N >= (double)n_pilot)) N = (double)n_pilot;
        if (N > (double)n_max) N = (double)n_max;
        begin[j] = n_pilot;
        extra[j] = (int64_t)N - n_pilot;
        total2 += extra[j];
        if (n_used) n_used[j] = (int64_t)N;
    }

    // phase 2: the remaining walks, paths n_pilot .. N-1 of each node
    if (total2 > 0) {
        L = choose_launch(ctx, cfg, dt, total2);
        WalkArgs A2 = base_args(ctx, L, dt, seed);
        A2.nodes = A.nodes;
        A2.node_ids = A.node_ids;
        Plan P2 = plan_ranges(n_nodes, begin.data(), extra.data(), L.chunk);
        st = run_phase(ctx, P2, L, A2, n_nodes, s2, v2, c2, &ms2);
        if (st != SDD_OK) return st;
    } else {
        s2.assign(s1.size(), 0.0);
        v2.assign(n_nodes, 0);
        c2[0] = c2[1] = c2[2] = 0;
    }
    for (int j = 0; j < n_nodes; ++j)
        for (int e = 0; e < E; ++e) {
            const size_t o = ((size_t)j * E + e) * 4;
            double q[4];
            for (int k = 0; k < 4; ++k) q[k] = s1[o + k] + s2[o + k];
            finish(q, v1[j] + v2[j], mean + ((size_t)j * E + e) * 2, se + ((size_t)j * E + e) * 2);
        }
    ctx->plan_valid = false;
    if (stats) {
        stats->steps = c1[0] + c2[0];
        stats->walks = c1[1] + c2[1];
        stats->truncated = c1[2] + c2[2];
        stats->kernel_ms = (double)ms1 + (double)ms2;
        stats->launches = total2 > 0 ? 4 : 2;
        stats->items = (int32_t)P1.items.size();
        stats->grid = L.grid;
        stats->block = L.block;
        stats->h2d_bytes = (uint64_t)n_nodes * 2 * sizeof(double);
        stats->d2h_bytes = (uint64_t)(s1.size() * 8 + n_nodes * 8) * (total2 > 0 ? 2 : 1);
    }
    return (c1[2] + c2[2]) ? SDD_E_TRUNCATED : SDD_OK;
}
