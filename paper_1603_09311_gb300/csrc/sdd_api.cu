// C ABI of libsdd: argument checks, model upload, work-item planning, the
// persistent walk launch and the fixed-order per-node reduction.
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <map>
#include <mutex>
#include <thread>
#include <string>
#include <vector>

#include "../../include/sdd.h"
#include "sdd_internal.cuh"

using namespace sdd;

void sdd::build_tiles(const int8_t *raster, int nx, int nz, std::vector<uint32_t> &coarse,
                      std::vector<uint8_t> &pool) {
    const int ntx = tile_cols(nx), ntz = tile_cols(nz);
    coarse.assign((size_t)ntx * ntz, 0u);
    pool.clear();
    uint8_t cells[kTile * kTile];
    for (int tz = 0; tz < ntz; ++tz)
        for (int tx = 0; tx < ntx; ++tx) {
            const int z0 = tz * kTile - kTile, x0 = tx * kTile - kTile;
            if (z0 >= 0 && z0 + kTile <= nz && x0 >= 0 && x0 + kTile <= nx) {
                for (int a = 0; a < kTile; ++a)
                    std::memcpy(cells + a * kTile, raster + (size_t)(z0 + a) * nx + x0, kTile);
            } else {  // a tile over the raster's edge: cells outside repeat the nearest edge cell
                for (int a = 0; a < kTile; ++a)
                    for (int b = 0; b < kTile; ++b) {
                        const int iz = std::min(std::max(z0 + a, 0), nz - 1);
                        const int ix = std::min(std::max(x0 + b, 0), nx - 1);
                        cells[a * kTile + b] = (uint8_t)raster[(size_t)iz * nx + ix];
                    }
            }
            uint64_t w[kTile * kTile / 8];
            std::memcpy(w, cells, sizeof(w));
            const uint64_t rep = 0x0101010101010101ull * cells[0];
            bool uniform = true;
            for (int k = 0; k < kTile * kTile / 8; ++k) uniform = uniform && w[k] == rep;
            if (uniform) {
                coarse[(size_t)tz * ntx + tx] = kTileUniform | cells[0];
            } else {
                coarse[(size_t)tz * ntx + tx] = (uint32_t)(pool.size() / (kTile * kTile));
                pool.insert(pool.end(), cells, cells + kTile * kTile);
            }
        }
}

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

// Work items of a call.  items are node by node, each node's in path order
// (the order in which the per-node sums add them); order[q] is the item the
// queue hands out q-th (empty: items in table order).
struct Plan {
    std::vector<Item> items;
    std::vector<int32_t> node_item0;  // [n_nodes + 1]
    std::vector<int32_t> order;
    std::vector<int32_t> qbase;       // grouped launches: [queues + 1] offsets into order
    std::vector<float> home_cut;      // grouped launches: [queues + 1] CTA shares
    long long total_paths = 0;
    bool cached = false;     // identical to the table already on the device
};

// What a plan was made from (the device copy is reused for an equal key).
struct PlanKey {
    std::vector<int64_t> paths;
    int chunk = -1, factor = 0;
    long long warps = 0;
    uint32_t offset = 0;
    bool operator==(const PlanKey &o) const {
        return chunk == o.chunk && factor == o.factor && warps == o.warps && offset == o.offset &&
               paths == o.paths;
    }
};

}  // namespace

struct sdd_ctx {
    int device = 0;
    int n_sm = 0;
    ModelDev M;
    int K = 0, E = 0;
    int geo = GEO_SHAPES;
    DevBuf raster, tiles;
    // per-call scratch
    DevBuf items, slots, trunc, counters, queue, err, nodes, node_ids, mean, se;
    DevBuf rec_steps, rec_counts, rec_occ, rec_hits, rec_exit, rec_wall, rec_mlast;
    DevBuf batch_models;  // model table of batched launches owned by this context
    DevBuf red_index;     // node -> first range of the range reduction (sdd_reduce_sums)
    std::vector<int32_t> h_red_index;
    Item *h_items = nullptr;  // pinned staging of the item table
    size_t h_items_cap = 0;
    cudaEvent_t items_done = nullptr;  // last copy out of h_items finished
    cudaStream_t stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // the plan whose item table was last uploaded (reused by a call with the
    // same key)
    Plan plan;
    PlanKey plan_key;
    bool plan_valid = false;
    uint64_t last_h2d = 0;
    cudaGraphExec_t graph_exec = nullptr;  // device work of the last graph-mode call
    uint64_t graph_updates = 0, graph_instantiations = 0;
    int tune_block = 0, tune_k = 0;        // autotuned threads per CTA, guided factor (0: none)
    bool tune_file_read = false;
    std::mutex submit_mu;                  // asynchronous requests may be submitted from several threads
};

namespace {

// Cap on the steps of one walk: keeps the occupation power sums (up to
// 27 x steps for four materials) inside 32 bits.  Caps are rounded up to a
// multiple of 8 (the steps of one iteration of the single-precision walk),
// in both precisions so that they truncate alike.
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
    const bool tm = m->diffusion != nullptr;
    for (int i = 0; i < m->n_eval * m->n_materials; ++i)
        if (!std::isfinite(m->kappa[i]) || (!tm && m->kappa[i] < 0.0))
            return fail(SDD_E_ARG, tm ? "kappa must be finite" : "kappa must be finite and >= 0");
    const int K = m->n_materials;
    if (tm) {
        for (int k = 0; k < K; ++k)
            if (!(m->diffusion[k] > 0.0) || !std::isfinite(m->diffusion[k]))
                return fail(SDD_E_ARG, "TM diffusion must be finite and > 0");
        if (K > 1 && !m->interfaces) return fail(SDD_E_ARG, "TM interfaces is NULL");
        for (int k = 0; k + 1 < K; ++k) {
            const double xk = m->interfaces[k];
            if (!(xk > d.x_min && xk < d.x_max) || (k > 0 && !(xk > m->interfaces[k - 1])))
                return fail(SDD_E_ARG, "TM interfaces must increase strictly inside (x_min, x_max)");
        }
        if (m->raster || m->n_shapes != 0) return fail(SDD_E_ARG, "TM mode takes no shapes or raster");
        if (m->g_kind != SDD_G_AFFINE && m->g_kind != SDD_G_X2MZ2 && m->g_kind != SDD_G_TM_COSH &&
            m->g_kind != SDD_G_TM_FLUX)
            return fail(SDD_E_ARG, "TM mode g_kind must be AFFINE, X2MZ2, TM_COSH or TM_FLUX");
        return SDD_OK;
    }
    if (m->raster) {
        if (m->nx < 1 || m->nz < 1 || m->nx > kMaxRasterSide || m->nz > kMaxRasterSide ||
            (long long)m->nx * m->nz > (1ll << 31))
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
    if (m->g_kind < SDD_G_COLUMNS || m->g_kind > SDD_G_X2MZ2)
        return fail(SDD_E_ARG, "unknown g_kind (TM_COSH and TM_FLUX need TM mode)");
    if (m->g_kind == SDD_G_COLUMNS &&
        (m->g_left < 0 || m->g_left >= K || m->g_right < 0 || m->g_right >= K))
        return fail(SDD_E_ARG, "g_left / g_right out of range");
    return SDD_OK;
}

// Side of the surface on which a triangle's single-precision test can
// accept a point: 0 the earth (every accepted point has Z >= fzs), 1 the air
// (every accepted point has Z < fzs), -1 neither or not decided.  The test
// is three edge functions fmaf(A, X, fmaf(B, Z, C)) >= 0 with float
// coefficients over points of the domain (|X| <= hw, |Z| <= hh); each is
// within 2^-23 (|A| hw + |B| hh + |C|) of its exact value, so an accepted
// point lies in the triangle whose edges are moved out by that bound
// (taken 8 times larger here).  That triangle's vertices decide.
static int triangle_side(const sdd::ShapeDev &S, float hw, float hh, float fzs) {
    double a[3], b[3], c[3];
    for (int e = 0; e < 3; ++e) {
        a[e] = S.f[3 * e];
        b[e] = S.f[3 * e + 1];
        c[e] = S.f[3 * e + 2];
        const double eps = std::ldexp(1.0, -20) * (std::fabs(a[e]) * hw + std::fabs(b[e]) * hh + std::fabs(c[e]));
        c[e] += eps;
    }
    double zmin = 1e300, zmax = -1e300;
    for (int e = 0; e < 3; ++e) {
        const int f = (e + 1) % 3;
        const double det = a[e] * b[f] - a[f] * b[e];
        if (!(std::fabs(det) > 1e-12 * (std::fabs(a[e] * b[f]) + std::fabs(a[f] * b[e]))) || det == 0.0)
            return -1;
        // a x + b z = -c for edges e and f
        const double z = (-a[e] * c[f] + a[f] * c[e]) / det;
        zmin = std::min(zmin, z);
        zmax = std::max(zmax, z);
    }
    const double margin = 1e-6 * (double)hh;
    if (zmin >= (double)fzs + margin) return 0;
    if (zmax < (double)fzs - margin) return 1;
    return -1;
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
    if (m->diffusion) {
        M.tm = 1;
        M.gcode = GC_TM;
        for (int k = 0; k < M.K; ++k) {
            M.diff[k] = m->diffusion[k];
            M.fdiff[k] = (float)m->diffusion[k];
            M.xif[k] = k + 1 < M.K ? m->interfaces[k] : d.x_max;
            M.fxif[k] = (float)M.xif[k];
        }
        for (int e = 0; e < M.E; ++e)
            for (int k = 0; k < M.K; ++k) {
                const std::complex<double> a =
                    std::sqrt(std::complex<double>(0.0, m->kappa[e * M.K + k] / m->diffusion[k]));
                M.tm_a[e][k][0] = a.real();
                M.tm_a[e][k][1] = a.imag();
            }
    } else if (!m->raster) {
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
        M.shape_air = 0;
        if (M.gcode == GC_RECT1) {
            // a vertical contact: the rectangle is the whole earth right of x0
            const sdd_shape &S = m->shapes[0];
            if (S.v[1] >= d.x_max && S.v[2] == 0.0 && S.v[3] >= d.z_max &&
                (float)(S.v[1] - M.xc) >= M.fhw && (float)(S.v[3] - M.zc) >= M.fhh) {
                M.gcode = GC_CONTACT;
            } else if (M.shapes[0].f[2] >= M.fzs) {
                // every point the single-precision test puts inside has
                // Z >= f[2] >= fzs: the rectangle is in the earth
            } else if (M.shapes[0].f[3] <= M.fzs) {
                M.shape_air = 1;  // Z < f[3] <= fzs: in the air
            } else {
                M.gcode = GC_SHAPES4;  // straddles the surface
            }
        } else if (M.gcode == GC_TRI1) {
            const int side = triangle_side(M.shapes[0], M.fhw, M.fhh, M.fzs);
            if (side == 0) M.shape_air = 0;
            else if (side == 1) M.shape_air = 1;
            else M.gcode = GC_SHAPES4;  // across or too near the surface
        }
    } else {
        M.gcode = GC_RASTER;
        M.nx = m->nx;
        M.nz = m->nz;
        M.sx = (double)m->nx / (d.x_max - d.x_min);
        M.sz = (double)m->nz / (d.z_max - d.z_min);
        M.fsx = (float)M.sx;
        M.fsz = (float)M.sz;
        M.fox = (float)(M.hw * M.sx - 0.5 + kTile);
        M.foz = (float)(M.hh * M.sz - 0.5 + kTile);
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
        if (cfg->guided_factor < 0 || cfg->guided_factor > 64)
            return fail(SDD_E_ARG, "guided_factor must be in 0..64");
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
    int kmax, block, grid;
    int chunk;   // > 0: fixed items of chunk paths; 0: guided
    int factor;  // guided: an item takes about 1 / (factor x warps) of the queued paths
    int64_t max_steps;
};

// Key of a launch shape in the tuning cache file: device, lookup program,
// materials bound, evaluations, precision and the decade of dt.
std::string tune_key(const sdd_ctx *ctx, int kmax, int gcode, bool f64, double dt) {
    char b[160];
    std::snprintf(b, sizeof(b), "sm%d gc%d k%d e%d p%d dt%d", ctx->n_sm, gcode, kmax, ctx->E, f64 ? 1 : 0,
                  (int)std::floor(std::log10(dt)));
    return b;
}

// The tuned shape for this context from SDD_TUNE_CACHE (read once).
void tune_from_file(sdd_ctx *ctx, int kmax, int gcode, bool f64, double dt) {
    if (ctx->tune_file_read) return;
    ctx->tune_file_read = true;
    const char *path = std::getenv("SDD_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    const std::string key = tune_key(ctx, kmax, gcode, f64, dt);
    char line[256];
    while (std::fgets(line, sizeof(line), f)) {
        int blk = 0, k = 0;
        const char *bar = std::strchr(line, '|');
        if (!bar) continue;
        if (std::string(line, bar - line) == key && std::sscanf(bar + 1, "%d %d", &blk, &k) == 2 &&
            blk >= 32 && blk <= 256 && blk % 32 == 0 && k >= 1 && k <= 64) {
            ctx->tune_block = blk;
            ctx->tune_k = k;
        }
    }
    std::fclose(f);
}

Launch choose_launch(const sdd_ctx *ctx, const sdd_config *cfg, double dt,
                     int kmax_override = 0, int gcode_override = -1) {
    Launch L;
    L.f64 = cfg && cfg->precision == SDD_FP64;
    L.kmax = kmax_override ? kmax_override : kmax_for(ctx->K);
    if (gcode_override < 0)
        tune_from_file(const_cast<sdd_ctx *>(ctx), L.kmax, ctx->M.gcode, L.f64, dt);
    const bool tuned = gcode_override < 0 && ctx->tune_block > 0;
    L.block = (cfg && cfg->block_threads) ? cfg->block_threads : (tuned ? ctx->tune_block : 256);
    L.factor = (cfg && cfg->guided_factor) ? cfg->guided_factor : (tuned ? ctx->tune_k : 2);
    const int gcode = gcode_override >= 0 ? gcode_override : ctx->M.gcode;
    int occ = L.f64 ? occupancy_f64(L.kmax, ctx->geo, L.block, ctx->E, ctx->K)
                    : occupancy_f32(L.kmax, gcode, L.block, ctx->E, std::max(ctx->K, L.kmax));
    if (occ < 1) occ = 1;
    if (cfg && cfg->ctas_per_sm > 0 && cfg->ctas_per_sm < occ) occ = cfg->ctas_per_sm;
    L.grid = ctx->n_sm * occ;
    L.chunk = (cfg && cfg->chunk_paths) ? cfg->chunk_paths : 0;
    L.max_steps = (cfg && cfg->max_steps) ? cfg->max_steps : (int64_t)std::ceil(20.0 / dt);
    if (L.max_steps > kMaxSteps) L.max_steps = kMaxSteps;
    L.max_steps = (L.max_steps + 7) / 8 * 8;  // single-precision walks advance 8 steps per iteration
    return L;
}

// Guided cuts of the paths of `nodes` (count[j] each): the sequence (node, k
// = the node's item index, size) in the order the queue hands the items out,
// sizes shrinking from about R / WF toward cmin (R the paths not yet cut, WF
// the warps x the guided factor).  In rounds, every node with paths left gets
// one item of the round's size.  When a round would take every node whole
// (many nodes, each with fewer paths than the round's size), the size is
// recomputed after every cut instead, nodes in turn, so that the last part of
// the queue still shrinks toward one walk per lane.
struct Cut {
    int32_t node, k, count;
};

void guided_cuts(const std::vector<int32_t> &nodes, const int64_t *count, long long WF, long long cmin,
                 std::vector<int32_t> &per_node, std::vector<Cut> &seq) {
    std::vector<int32_t> live;
    long long R = 0, cmax = 0;
    for (int32_t j : nodes)
        if (count[j] > 0) {
            live.push_back(j);
            R += count[j];
            cmax = std::max<long long>(cmax, count[j]);
        }
    auto size = [&](long long rem) {
        long long c = (rem + WF - 1) / WF;
        c = std::max(cmin, (c + 31) / 32 * 32);
        return std::min<long long>(c, 1 << 24);
    };
    std::vector<int64_t> left(live.size());
    for (size_t i = 0; i < live.size(); ++i) left[i] = count[live[i]];
    if (size(R) >= cmax && live.size() > 1) {
        // one cut at a time, nodes in turn
        size_t at = 0, n_live = live.size();
        while (n_live > 0) {
            while (left[at] == 0) at = at + 1 == live.size() ? 0 : at + 1;
            const int64_t take = std::min<int64_t>(size(R), left[at]);
            const int32_t j = live[at];
            seq.push_back({j, per_node[j]++, (int32_t)take});
            left[at] -= take;
            R -= take;
            if (left[at] == 0) --n_live;
            at = at + 1 == live.size() ? 0 : at + 1;
        }
        return;
    }
    while (!live.empty()) {
        const long long c = size(R);
        size_t keep = 0;
        for (size_t i = 0; i < live.size(); ++i) {
            const int32_t j = live[i];
            const int64_t take = std::min<int64_t>(c, left[i]);
            seq.push_back({j, per_node[j]++, (int32_t)take});
            left[i] -= take;
            R -= take;
            if (left[i] > 0) {
                live[keep] = j;
                left[keep] = left[i];
                ++keep;
            }
        }
        live.resize(keep);
        left.resize(keep);
    }
}

// Items for paths [offset + begin[j], offset + begin[j] + count[j]) of every
// node j (begin == nullptr: from 0), for the launch L.
//   Fixed (L.chunk > 0): items of L.chunk paths, node by node.
//   Guided (L.chunk == 0): cut in rounds; in each round every node with paths
//   left gets one item of c = ceil(R / (F W)) paths, rounded up to a multiple
//   of 32 and at least 32 (or at least total / 2^20, which bounds the table),
//   R being the paths not yet cut, W the warps of the grid and F = L.factor.
//   The queue hands items out in the order they were cut, so sizes shrink
//   from about R / (F W) to one walk per lane toward the end of the queue,
//   and no warp takes a large item just before the queue runs dry.
Plan plan_work(int32_t n_nodes, const int64_t *begin, const int64_t *count, uint32_t p_offset,
               const Launch &L) {
    Plan P;
    P.node_item0.assign((size_t)n_nodes + 1, 0);
    for (int j = 0; j < n_nodes; ++j) P.total_paths += count[j];
    auto first = [&](int j) -> int64_t { return begin ? begin[j] : 0; };
    if (L.chunk > 0) {
        for (int j = 0; j < n_nodes; ++j) {
            P.node_item0[j] = (int32_t)P.items.size();
            for (int64_t p = 0; p < count[j]; p += L.chunk) {
                Item I;
                I.node = j;
                I.path0 = p_offset + (uint32_t)(first(j) + p);
                I.count = (int32_t)std::min<int64_t>(L.chunk, count[j] - p);
                I.model = 0;
                P.items.push_back(I);
            }
        }
        P.node_item0[n_nodes] = (int32_t)P.items.size();
        return P;
    }
    const long long W = std::max<long long>(1, (long long)L.grid * (L.block / 32) * std::max(L.factor, 1));
    const long long cmin = std::max<long long>(32, (P.total_paths / (1 << 20) + 31) / 32 * 32);
    std::vector<Cut> seq;
    std::vector<int32_t> all((size_t)n_nodes), per_node((size_t)n_nodes, 0);
    std::vector<int64_t> done((size_t)n_nodes, 0);
    for (int j = 0; j < n_nodes; ++j) all[j] = j;
    guided_cuts(all, count, W, cmin, per_node, seq);
    for (int j = 0; j < n_nodes; ++j) P.node_item0[j + 1] = P.node_item0[j] + per_node[j];
    P.items.resize(seq.size());
    P.order.resize(seq.size());
    std::fill(done.begin(), done.end(), 0);
    for (size_t q = 0; q < seq.size(); ++q) {
        const Cut &x = seq[q];
        const int32_t idx = P.node_item0[x.node] + x.k;
        Item &I = P.items[idx];
        I.node = x.node;
        I.path0 = p_offset + (uint32_t)(first(x.node) + done[x.node]);
        I.count = x.count;
        I.model = 0;
        done[x.node] += x.count;
        P.order[q] = idx;
    }
    return P;
}

// Items of a launch over several models, one queue per model (the models of
// a batched or served launch each have their own tile map; keeping an SM on
// few models keeps their tile maps in its L1).  Model m's nodes are cut with
// the guided sizes of plan_work for the warps of its share of the grid (its
// share of the walks), the queue of model m hands its items out in cut
// order, and CTAs are homed on the queues in proportion to the shares.  The
// item table stays node by node (the per-node sums add items in path order).
Plan plan_grouped(int32_t n_nodes, const int64_t *begin, const int64_t *count, const int32_t *node_model,
                  int32_t n_models, const Launch &L) {
    Plan P;
    P.node_item0.assign((size_t)n_nodes + 1, 0);
    std::vector<long long> walks((size_t)n_models, 0);
    for (int j = 0; j < n_nodes; ++j) {
        P.total_paths += count[j];
        walks[node_model[j]] += count[j];
    }
    auto first = [&](int j) -> int64_t { return begin ? begin[j] : 0; };
    const long long Wall = std::max<long long>(1, (long long)L.grid * (L.block / 32));
    const long long F = std::max(L.factor, 1);
    const long long cmin = std::max<long long>(32, (P.total_paths / (1 << 20) + 31) / 32 * 32);
    std::vector<std::vector<int32_t>> nodes_of((size_t)n_models);
    for (int j = 0; j < n_nodes; ++j) nodes_of[node_model[j]].push_back(j);
    std::vector<std::vector<Cut>> seq((size_t)n_models);
    std::vector<int32_t> per_node((size_t)n_nodes, 0);
    std::vector<int64_t> done((size_t)n_nodes, 0);
    P.home_cut.assign((size_t)n_models + 1, 0.f);
    long long acc = 0;
    for (int m = 0; m < n_models; ++m) {
        P.home_cut[m] = P.total_paths ? (float)((double)acc / (double)P.total_paths) : 0.f;
        acc += walks[m];
        const long long W = std::max<long long>(1, (long long)std::llround((double)Wall * walks[m] /
                                                                          std::max<double>(1.0, (double)P.total_paths))) * F;
        guided_cuts(nodes_of[m], count, W, cmin, per_node, seq[m]);
    }
    P.home_cut[n_models] = 1.f;
    for (int j = 0; j < n_nodes; ++j) P.node_item0[j + 1] = P.node_item0[j] + per_node[j];
    const size_t ni = (size_t)P.node_item0[n_nodes];
    P.items.resize(ni);
    P.order.reserve(ni);
    P.qbase.assign((size_t)n_models + 1, 0);
    std::fill(done.begin(), done.end(), 0);
    for (int m = 0; m < n_models; ++m) {
        P.qbase[m] = (int32_t)P.order.size();
        for (const Cut &x : seq[m]) {
            const int32_t idx = P.node_item0[x.node] + x.k;
            Item &I = P.items[idx];
            I.node = x.node;
            I.path0 = (uint32_t)(first(x.node) + done[x.node]);
            I.count = x.count;
            I.model = m;
            done[x.node] += x.count;
            P.order.push_back(idx);
        }
    }
    P.qbase[n_models] = (int32_t)P.order.size();
    return P;
}

// The plan of a call with per-node path counts n_paths (paths from p_offset),
// reusing the context's last plan, and its device table, for an equal key.
const Plan &plan_cached(sdd_ctx *ctx, int32_t n_nodes, const int64_t *n_paths, uint32_t p_offset,
                        const Launch &L) {
    PlanKey key;
    key.paths.assign(n_paths, n_paths + n_nodes);
    key.chunk = L.chunk;
    key.factor = L.chunk > 0 ? 0 : L.factor;
    key.warps = L.chunk > 0 ? 0 : (long long)L.grid * (L.block / 32);
    key.offset = p_offset;
    if (ctx->plan_valid && key == ctx->plan_key) {
        ctx->plan.cached = true;
        return ctx->plan;
    }
    // the device table becomes valid for this key only once its upload is queued
    ctx->plan_valid = false;
    ctx->plan = plan_work(n_nodes, nullptr, n_paths, p_offset, L);
    ctx->plan.cached = false;
    ctx->plan_key = std::move(key);
    return ctx->plan;
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

// Scratch buffers and the item table of a plan: items, node_item0 and the
// queue order, uploaded through pinned staging unless the device already
// holds this plan.
size_t table_bytes(const Plan &P, int n_nodes) {
    return P.items.size() * sizeof(Item) + ((size_t)n_nodes + 1) * sizeof(int32_t) +
           P.order.size() * sizeof(int32_t) + P.qbase.size() * sizeof(int32_t) +
           P.home_cut.size() * sizeof(float);
}

// The item table as uploaded: items, node_item0, order, then (grouped
// launches) qbase and home_cut.
void pack_table(const Plan &P, int n_nodes, unsigned char *h) {
    const size_t ni = P.items.size();
    std::memcpy(h, P.items.data(), ni * sizeof(Item));
    h += ni * sizeof(Item);
    std::memcpy(h, P.node_item0.data(), ((size_t)n_nodes + 1) * sizeof(int32_t));
    h += ((size_t)n_nodes + 1) * sizeof(int32_t);
    if (!P.order.empty()) std::memcpy(h, P.order.data(), P.order.size() * sizeof(int32_t));
    h += P.order.size() * sizeof(int32_t);
    if (!P.qbase.empty()) std::memcpy(h, P.qbase.data(), P.qbase.size() * sizeof(int32_t));
    h += P.qbase.size() * sizeof(int32_t);
    if (!P.home_cut.empty()) std::memcpy(h, P.home_cut.data(), P.home_cut.size() * sizeof(float));
}

// Device pointers of a packed table at d: order, qbase, home_cut and the
// number of queues.
void table_args(const Plan &P, int n_nodes, const unsigned char *d, WalkArgs &A) {
    const size_t ni = P.items.size();
    const unsigned char *o = d + ni * sizeof(Item) + ((size_t)n_nodes + 1) * sizeof(int32_t);
    A.order = P.order.empty() ? nullptr : reinterpret_cast<const int32_t *>(o);
    o += P.order.size() * sizeof(int32_t);
    A.qbase = P.qbase.empty() ? nullptr : reinterpret_cast<const int32_t *>(o);
    o += P.qbase.size() * sizeof(int32_t);
    A.home_cut = P.home_cut.empty() ? nullptr : reinterpret_cast<const float *>(o);
    A.n_queues = P.qbase.empty() ? 1 : (int32_t)P.qbase.size() - 1;
}

sdd_status prepare(sdd_ctx *ctx, const Plan &P, int n_nodes, cudaStream_t s) {
    const size_t ni = P.items.size();
    if (ni == 0) return SDD_OK;
    const size_t hbytes = table_bytes(P, n_nodes);
    SDD_CUDA(ctx->items.ensure(hbytes));
    SDD_CUDA(ctx->slots.ensure(ni * (size_t)ctx->E * 4 * sizeof(double)));
    SDD_CUDA(ctx->trunc.ensure(ni * sizeof(int32_t)));
    SDD_CUDA(ctx->counters.ensure(3 * sizeof(unsigned long long)));
    SDD_CUDA(ctx->queue.ensure(std::max<size_t>(P.qbase.size(), 1) * sizeof(int32_t)));
    SDD_CUDA(ctx->err.ensure(sizeof(int32_t)));
    ctx->last_h2d = 0;
    const bool own = &P == &ctx->plan;
    if (!(own && P.cached)) {
        if (ctx->items_done) SDD_CUDA(cudaEventSynchronize(ctx->items_done));
        if (hbytes > ctx->h_items_cap) {
            if (ctx->h_items) cudaFreeHost(ctx->h_items);
            ctx->h_items = nullptr;
            ctx->h_items_cap = 0;
            SDD_CUDA(cudaMallocHost((void **)&ctx->h_items, hbytes + hbytes / 4 + 256));
            ctx->h_items_cap = hbytes + hbytes / 4 + 256;
        }
        pack_table(P, n_nodes, reinterpret_cast<unsigned char *>(ctx->h_items));
        SDD_CUDA(cudaMemcpyAsync(ctx->items.p, ctx->h_items, hbytes, cudaMemcpyHostToDevice, s));
        SDD_CUDA(cudaEventRecord(ctx->items_done, s));
        ctx->last_h2d = hbytes;
        ctx->plan_valid = own;
    }
    return SDD_OK;
}

// Device work of a prepared plan: clear counters, walk, reduce.
sdd_status enqueue(sdd_ctx *ctx, const Plan &P, const Launch &L, WalkArgs A, cudaStream_t s,
                   bool timed, bool do_reduce, double *d_mean, double *d_se, int n_nodes,
                   const ModelDev *model = nullptr) {
    const ModelDev &MD = model ? *model : ctx->M;
    const size_t ni = P.items.size();
    if (ni == 0) return SDD_OK;
    SDD_CUDA(cudaMemsetAsync(ctx->queue.p, 0, std::max<size_t>(P.qbase.size(), 1) * sizeof(int32_t), s));
    SDD_CUDA(cudaMemsetAsync(ctx->counters.p, 0, 3 * sizeof(unsigned long long), s));
    A.items = (const Item *)ctx->items.p;
    A.n_items = (int32_t)ni;
    table_args(P, n_nodes, reinterpret_cast<const unsigned char *>(ctx->items.p), A);
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
    cudaError_t e = L.f64 ? launch_walk_f64(L.kmax, ctx->geo, MD, A, grid, L.block, s)
                          : launch_walk_f32(L.kmax, ctx->geo, MD, A, grid, L.block, s);
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

sdd_status run(sdd_ctx *ctx, const Plan &P, const Launch &L, WalkArgs A, cudaStream_t s,
               bool timed, bool do_reduce, double *d_mean, double *d_se, int n_nodes,
               const ModelDev *model = nullptr) {
    sdd_status st = prepare(ctx, P, n_nodes, s);
    if (st != SDD_OK) return st;
    return enqueue(ctx, P, L, A, s, timed, do_reduce, d_mean, d_se, n_nodes, model);
}

}  // namespace

int sdd::report_error(int status, const char *msg) { return (int)fail((sdd_status)status, msg); }

int sdd::ctx_site_diffusion(const sdd_ctx *c, double x, double *D) {
    if (!c || c->geo != GEO_TM) return 0;
    int m = 0;
    while (m < c->K - 1 && x >= c->M.xif[m]) ++m;
    *D = c->M.diff[m];
    return 1;
}

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
    if (model->diffusion) c->geo = GEO_TM;
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
        std::vector<uint32_t> coarse;
        std::vector<uint8_t> pool;
        build_tiles(model->raster, model->nx, model->nz, coarse, pool);
        const size_t cb = (coarse.size() * sizeof(uint32_t) + 255) / 256 * 256;
        e = c->tiles.ensure(cb + pool.size() + 16);
        if (e == cudaSuccess)
            e = cudaMemcpy(c->tiles.p, coarse.data(), coarse.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !pool.empty())
            e = cudaMemcpy((unsigned char *)c->tiles.p + cb, pool.data(), pool.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            sdd_destroy(c);
            return e == cudaErrorMemoryAllocation ? fail(SDD_E_OOM, "tile map allocation")
                                                  : cuda_fail(e, "tile map upload");
        }
        c->M.tcoarse = (const uint32_t *)c->tiles.p;
        c->M.tpool = (const uint8_t *)c->tiles.p + cb;
        c->M.ntx = tile_cols(model->nx);
        c->M.tpool_off = (uint32_t)cb;
    }
    *out = c;
    return SDD_OK;
}

void sdd_destroy(sdd_ctx *c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    DevBuf *bufs[] = {&c->raster, &c->tiles, &c->items, &c->slots, &c->trunc, &c->counters, &c->queue,
                      &c->err, &c->nodes, &c->node_ids, &c->mean, &c->se, &c->rec_steps,
                      &c->rec_counts, &c->rec_occ, &c->rec_hits, &c->rec_exit, &c->rec_wall,
                      &c->rec_mlast,
                      &c->batch_models, &c->red_index};
    for (DevBuf *b : bufs) b->release();
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->h_items) cudaFreeHost(c->h_items);
    if (c->items_done) cudaEventDestroy(c->items_done);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

int32_t sdd_n_eval(const sdd_ctx *c) { return c ? c->E : 0; }
int32_t sdd_n_materials(const sdd_ctx *c) { return c ? c->K : 0; }

static_assert(SDD_PROGRAM_LAYERS == GC_LAYER && SDD_PROGRAM_RECT == GC_RECT1 &&
                  SDD_PROGRAM_TRIANGLE == GC_TRI1 && SDD_PROGRAM_SHAPES4 == GC_SHAPES4 &&
                  SDD_PROGRAM_SHAPES16 == GC_SHAPES16 && SDD_PROGRAM_RASTER == GC_RASTER &&
                  SDD_PROGRAM_CONTACT == GC_CONTACT && SDD_PROGRAM_TM == GC_TM,
              "lookup program codes of the header and of the walk differ");

sdd_status sdd_model_program(const sdd_model_desc *model, int32_t *program, int32_t *shape_side) {
    if (!program) return fail(SDD_E_ARG, "program is NULL");
    const sdd_status st = check_model(model);
    if (st != SDD_OK) return st;
    std::unique_ptr<ModelDev> M(new (std::nothrow) ModelDev());
    if (!M) return fail(SDD_E_OOM, "host allocation failed");
    build_model(model, *M);
    *program = M->gcode;
    if (shape_side) {
        const bool one = M->gcode == GC_RECT1 || M->gcode == GC_TRI1 || M->gcode == GC_CONTACT;
        *shape_side = one ? M->shape_air : -1;
    }
    return SDD_OK;
}

sdd_status sdd_plan_items(int32_t n_nodes, const int64_t *n_paths, int32_t warps, int32_t guided_factor,
                          int32_t chunk_paths, int32_t max_items, int32_t *node, uint32_t *path0,
                          int32_t *count, int32_t *n_items) {
    if (!n_items) return fail(SDD_E_ARG, "n_items is NULL");
    *n_items = 0;
    if (n_nodes < 0 || (n_nodes > 0 && !n_paths)) return fail(SDD_E_ARG, "bad nodes / n_paths");
    if (warps < 1 || guided_factor < 1 || chunk_paths < 0 || max_items < 0)
        return fail(SDD_E_ARG, "warps and guided_factor must be >= 1, chunk_paths and max_items >= 0");
    for (int32_t j = 0; j < n_nodes; ++j)
        if (n_paths[j] < 0 || n_paths[j] > 0xffffffffLL) return fail(SDD_E_ARG, "path count out of range");
    Launch L{};
    L.grid = warps;
    L.block = 32;
    L.factor = guided_factor;
    L.chunk = chunk_paths;
    const Plan P = plan_work(n_nodes, nullptr, n_paths, 0, L);
    const int64_t n = (int64_t)P.items.size();
    if (n > 0x7fffffffLL) return fail(SDD_E_ARG, "too many items");
    *n_items = (int32_t)n;
    if (n > max_items) return fail(SDD_E_ARG, "more items than max_items");
    if (n > 0 && (!node || !path0 || !count)) return fail(SDD_E_ARG, "output pointer is NULL");
    for (int64_t q = 0; q < n; ++q) {
        const Item &I = P.items[P.order.empty() ? q : P.order[q]];
        node[q] = I.node;
        path0[q] = I.path0;
        count[q] = I.count;
    }
    return SDD_OK;
}

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
    const Launch L = choose_launch(ctx, cfg, dt);
    const Plan &P = plan_cached(ctx, n_nodes, n_paths, 0, L);
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
    const Launch L = choose_launch(ctx, cfg, dt);
    const Plan &P = plan_cached(ctx, n_nodes, n_paths, 0, L);
    cudaStream_t s = (cudaStream_t)stream;
    WalkArgs A = base_args(ctx, L, dt, seed);
    A.nodes = d_nodes_xz;
    A.node_ids = d_node_ids;
    if (!(cfg && cfg->use_graph)) {
        st = run(ctx, P, L, A, s, false, true, d_mean, d_se, n_nodes);
        if (st != SDD_OK) return st;
        if (d_counters)
            SDD_CUDA(cudaMemcpyAsync(d_counters, ctx->counters.p, 3 * sizeof(uint64_t),
                                     cudaMemcpyDeviceToDevice, s));
        return SDD_OK;
    }
    // graph mode: the item table goes up on the caller's stream; the device
    // work is captured on the context's stream into a graph, the cached
    // executable graph is updated in place (re-instantiated only when the
    // captured work changes shape) and launched on the caller's stream
    st = prepare(ctx, P, n_nodes, s);
    if (st != SDD_OK) return st;
    cudaGraph_t g = nullptr;
    SDD_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    st = enqueue(ctx, P, L, A, ctx->stream, false, true, d_mean, d_se, n_nodes);
    if (st == SDD_OK && d_counters) {
        cudaError_t e = cudaMemcpyAsync(d_counters, ctx->counters.p, 3 * sizeof(uint64_t),
                                        cudaMemcpyDeviceToDevice, ctx->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "counter copy");
    }
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
    if (st != SDD_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    bool updated = false;
    if (ctx->graph_exec) {
        cudaGraphExecUpdateResultInfo info;
        updated = cudaGraphExecUpdate(ctx->graph_exec, g, &info) == cudaSuccess;
        if (!updated) {
            cudaGetLastError();
            cudaGraphExecDestroy(ctx->graph_exec);
            ctx->graph_exec = nullptr;
        }
    }
    if (!updated) {
        e = cudaGraphInstantiate(&ctx->graph_exec, g, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            ctx->graph_exec = nullptr;
            return cuda_fail(e, "cudaGraphInstantiate");
        }
        ctx->graph_instantiations += 1;
    } else {
        ctx->graph_updates += 1;
    }
    cudaGraphDestroy(g);
    SDD_CUDA(cudaGraphLaunch(ctx->graph_exec, s));
    return SDD_OK;
}

}  // extern "C"

namespace {

// Per-path records of paths p0 .. p0+count-1 of one node (the walk kernel
// writes them instead of summing samples).
sdd_status walk_records(sdd_ctx *ctx, double x0, double z0, uint32_t node_id, uint32_t p0,
                        int32_t count, double dt, uint64_t seed, const sdd_config *cfg,
                        int64_t *steps, int64_t *counts, double *occ, double *exit_xzt,
                        int32_t *wall, int32_t *m_last, int64_t *hits) {
    const int64_t np = count;
    sdd_status st = check_call(ctx, count > 0 ? 1 : 0, &np, dt, cfg);
    if (st != SDD_OK) return st;
    if (count <= 0) return count == 0 ? SDD_OK : fail(SDD_E_ARG, "count < 0");
    if (!steps) return fail(SDD_E_ARG, "steps must not be NULL");
    if ((uint64_t)p0 + (uint64_t)count > 0x100000000ull) return fail(SDD_E_ARG, "path range overflows 32 bits");
    const double xz[2] = {x0, z0};
    st = check_nodes(ctx, xz, 1);
    if (st != SDD_OK) return st;
    const Launch L = choose_launch(ctx, cfg, dt);
    const Plan P = plan_work(1, nullptr, &np, p0, L);
    cudaStream_t s = ctx->stream;
    SDD_CUDA(ctx->nodes.ensure(2 * sizeof(double)));
    SDD_CUDA(ctx->node_ids.ensure(sizeof(uint32_t)));
    SDD_CUDA(ctx->rec_steps.ensure((size_t)count * 8));
    SDD_CUDA(ctx->rec_counts.ensure((size_t)count * ctx->K * 8));
    SDD_CUDA(ctx->rec_occ.ensure((size_t)count * ctx->K * 8));
    SDD_CUDA(ctx->rec_hits.ensure((size_t)count * 8));
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
    A.rec_occ = (double *)ctx->rec_occ.p;
    A.rec_hits = (int64_t *)ctx->rec_hits.p;
    A.rec_exit = (double *)ctx->rec_exit.p;
    A.rec_wall = (int32_t *)ctx->rec_wall.p;
    A.rec_mlast = (int32_t *)ctx->rec_mlast.p;
    st = run(ctx, P, L, A, s, false, false, nullptr, nullptr, 1);
    if (st != SDD_OK) return st;
    SDD_CUDA(cudaMemcpyAsync(steps, ctx->rec_steps.p, (size_t)count * 8, cudaMemcpyDeviceToHost, s));
    if (counts)
        SDD_CUDA(cudaMemcpyAsync(counts, ctx->rec_counts.p, (size_t)count * ctx->K * 8, cudaMemcpyDeviceToHost, s));
    if (occ) SDD_CUDA(cudaMemcpyAsync(occ, ctx->rec_occ.p, (size_t)count * ctx->K * 8, cudaMemcpyDeviceToHost, s));
    if (hits) SDD_CUDA(cudaMemcpyAsync(hits, ctx->rec_hits.p, (size_t)count * 8, cudaMemcpyDeviceToHost, s));
    if (exit_xzt)
        SDD_CUDA(cudaMemcpyAsync(exit_xzt, ctx->rec_exit.p, (size_t)count * 24, cudaMemcpyDeviceToHost, s));
    if (wall) SDD_CUDA(cudaMemcpyAsync(wall, ctx->rec_wall.p, (size_t)count * 4, cudaMemcpyDeviceToHost, s));
    if (m_last) SDD_CUDA(cudaMemcpyAsync(m_last, ctx->rec_mlast.p, (size_t)count * 4, cudaMemcpyDeviceToHost, s));
    SDD_CUDA(cudaStreamSynchronize(s));
    return SDD_OK;
}

}  // namespace

extern "C" sdd_status sdd_walk_records(sdd_ctx *ctx, double x0, double z0, uint32_t node_id, uint32_t p0,
                                       int32_t count, double dt, uint64_t seed, const sdd_config *cfg,
                                       int64_t *steps, int64_t *counts, double *exit_xzt, int32_t *wall,
                                       int32_t *m_last) {
    if (ctx && ctx->geo == GEO_TM)
        return fail(SDD_E_UNSUPPORTED, "TM walks split steps between strips: use sdd_walk_occupation");
    return walk_records(ctx, x0, z0, node_id, p0, count, dt, seed, cfg, steps, counts, nullptr,
                        exit_xzt, wall, m_last, nullptr);
}

extern "C" sdd_status sdd_walk_occupation(sdd_ctx *ctx, double x0, double z0, uint32_t node_id,
                                          uint32_t p0, int32_t count, double dt, uint64_t seed,
                                          const sdd_config *cfg, int64_t *steps, double *occ,
                                          double *exit_xzt, int32_t *wall, int32_t *m_last,
                                          int64_t *hits) {
    return walk_records(ctx, x0, z0, node_id, p0, count, dt, seed, cfg, steps, nullptr, occ, exit_xzt,
                        wall, m_last, hits);
}


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
// with that device current (the name is only a host-side stand-in).  Host
// threads may make their first calls at once: the cache is atomic, and two
// threads that both look the address up store the same value.
constexpr int kNaMaxDevices = 64;
std::atomic<unsigned char *> g_noalloc_ptr[kNaMaxDevices];

sdd_status noalloc_scratch(int device, unsigned char **out) {
    if (device < 0 || device >= kNaMaxDevices) return fail(SDD_E_UNSUPPORTED, "device id too large");
    unsigned char *p = g_noalloc_ptr[device].load(std::memory_order_acquire);
    if (!p) {
        void *a = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&a, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        p = static_cast<unsigned char *>(a);
        g_noalloc_ptr[device].store(p, std::memory_order_release);
    }
    *out = p;
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
            I.model = 0;
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
    if (cfg && cfg->use_graph)
        return fail(SDD_E_UNSUPPORTED, "sdd_interface_values_noalloc launches its kernels directly: "
                                       "cfg->use_graph must be 0");
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
    Launch L = choose_launch(ctx, cfg, dt);
    // fixed-size items (the table is built on the device): about 6 per warp,
    // widened until they fit the scratch array
    long long chunk = L.chunk;
    if (chunk == 0) {
        const long long per = (long long)L.grid * (L.block / 32) * 6;
        chunk = std::max<long long>(32, ((total + per - 1) / per + 31) / 32 * 32);
    }
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
// Path ranges (sdd_range_sums, sdd_range_sums_device) and the fixed-order
// reduction of their sums (sdd_reduce_sums, sdd_reduce_sums_device).
//
// The walks of a node are independent of one another, and so are the nodes
// (Sec. 5), so one evaluation can be cut into ranges (a node and a contiguous
// range of its paths) that separate processes evaluate.  A range's raw sums
// are those of its walks under the node's Philox streams; the node's mean and
// standard error follow from the sums of its ranges, added in range order.

namespace {

__global__ void range_reduce_kernel(const double *__restrict__ sums, const long long *__restrict__ n_valid,
                                    const int32_t *__restrict__ node_range0, int n_nodes, int E,
                                    double *__restrict__ mean, double *__restrict__ se) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_nodes * E) return;
    const int j = t / E, e = t % E;
    double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    long long nv = 0;
    for (int r = node_range0[j]; r < node_range0[j + 1]; ++r) {
        const double *o = sums + ((size_t)r * E + e) * 4;
        s0 += o[0]; s1 += o[1]; s2 += o[2]; s3 += o[3];
        nv += n_valid[r];
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

sdd_status check_ranges(sdd_ctx *ctx, int32_t n, const int64_t *begin, const int64_t *count, double dt,
                        const sdd_config *cfg) {
    sdd_status st = check_call(ctx, n, count, dt, cfg);
    if (st != SDD_OK) return st;
    if (n > 0 && !begin) return fail(SDD_E_ARG, "path_begin is NULL");
    for (int i = 0; i < n; ++i)
        if (begin[i] < 0 || begin[i] + count[i] > 0x100000000ll)
            return fail(SDD_E_ARG, "a path range must lie in 0..2^32");
    if (cfg && cfg->use_graph)
        return fail(SDD_E_UNSUPPORTED, "range sums launch their kernels directly: cfg->use_graph must be 0");
    return SDD_OK;
}

// Walks of the ranges and their raw sums into d_sums / d_n_valid (device).
sdd_status range_walks(sdd_ctx *ctx, const double *d_nodes, const uint32_t *d_ids, int32_t n,
                       const int64_t *begin, const int64_t *count, double dt, uint64_t seed,
                       const sdd_config *cfg, double *d_sums, long long *d_nv, cudaStream_t s,
                       bool timed, size_t *n_items) {
    const Launch L = choose_launch(ctx, cfg, dt);
    ctx->plan_valid = false;
    const Plan P = plan_work(n, begin, count, 0, L);
    WalkArgs A = base_args(ctx, L, dt, seed);
    A.nodes = d_nodes;
    A.node_ids = d_ids;
    sdd_status st = run(ctx, P, L, A, s, timed, false, nullptr, nullptr, n);
    if (st != SDD_OK) return st;
    const size_t ni = P.items.size();
    const Item *d_items = (const Item *)ctx->items.p;
    const int32_t *d_i0 = (const int32_t *)(reinterpret_cast<unsigned char *>(ctx->items.p) + ni * sizeof(Item));
    const int nt = n * ctx->E;
    sums_kernel<<<(nt + 127) / 128, 128, 0, s>>>((const double *)ctx->slots.p, (const int32_t *)ctx->trunc.p,
                                                d_items, d_i0, n, ctx->E, d_sums, d_nv);
    SDD_CUDA(cudaGetLastError());
    if (n_items) *n_items = ni;
    return SDD_OK;
}

// node -> first range (CSR) of a nondecreasing range -> node map.
sdd_status range_index(sdd_ctx *ctx, int32_t n_nodes, int32_t n_ranges, const int32_t *range_node) {
    if (n_nodes < 0 || n_ranges < 0) return fail(SDD_E_ARG, "n_nodes and n_ranges must be >= 0");
    if (n_ranges > 0 && !range_node) return fail(SDD_E_ARG, "range_node is NULL");
    std::vector<int32_t> &ix = ctx->h_red_index;
    ix.assign((size_t)n_nodes + 1, 0);
    for (int r = 0; r < n_ranges; ++r) {
        if (range_node[r] < 0 || range_node[r] >= n_nodes || (r > 0 && range_node[r] < range_node[r - 1]))
            return fail(SDD_E_ARG, "range_node must be nondecreasing node indices in 0..n_nodes-1");
        ix[(size_t)range_node[r] + 1] += 1;
    }
    for (int j = 0; j < n_nodes; ++j) ix[(size_t)j + 1] += ix[j];
    return SDD_OK;
}

}  // namespace

extern "C" sdd_status sdd_range_sums(sdd_ctx *ctx, const double *nodes_xz, const uint32_t *node_ids,
                                     int32_t n_ranges, const int64_t *path_begin,
                                     const int64_t *path_count, double dt, uint64_t seed,
                                     const sdd_config *cfg, double *sums, int64_t *n_valid,
                                     sdd_stats *stats) {
    sdd_status st = check_ranges(ctx, n_ranges, path_begin, path_count, dt, cfg);
    if (st != SDD_OK) return st;
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (n_ranges == 0) return SDD_OK;
    if (!nodes_xz || !sums || !n_valid) return fail(SDD_E_ARG, "nodes_xz, sums and n_valid must not be NULL");
    st = check_nodes(ctx, nodes_xz, n_ranges);
    if (st != SDD_OK) return st;
    cudaStream_t s = ctx->stream;
    const size_t sb = (size_t)n_ranges * ctx->E * 4 * sizeof(double);
    SDD_CUDA(ctx->nodes.ensure((size_t)n_ranges * 2 * sizeof(double)));
    SDD_CUDA(ctx->mean.ensure(sb));
    SDD_CUDA(ctx->se.ensure((size_t)n_ranges * sizeof(long long)));
    SDD_CUDA(cudaMemcpyAsync(ctx->nodes.p, nodes_xz, (size_t)n_ranges * 2 * sizeof(double),
                             cudaMemcpyHostToDevice, s));
    const uint32_t *d_ids = nullptr;
    if (node_ids) {
        SDD_CUDA(ctx->node_ids.ensure((size_t)n_ranges * sizeof(uint32_t)));
        SDD_CUDA(cudaMemcpyAsync(ctx->node_ids.p, node_ids, (size_t)n_ranges * sizeof(uint32_t),
                                 cudaMemcpyHostToDevice, s));
        d_ids = (const uint32_t *)ctx->node_ids.p;
    }
    size_t ni = 0;
    st = range_walks(ctx, (const double *)ctx->nodes.p, d_ids, n_ranges, path_begin, path_count, dt, seed,
                     cfg, (double *)ctx->mean.p, (long long *)ctx->se.p, s, true, &ni);
    if (st != SDD_OK) return st;
    unsigned long long cnt[3] = {0, 0, 0};
    SDD_CUDA(cudaMemcpyAsync(sums, ctx->mean.p, sb, cudaMemcpyDeviceToHost, s));
    SDD_CUDA(cudaMemcpyAsync(n_valid, ctx->se.p, (size_t)n_ranges * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SDD_CUDA(cudaMemcpyAsync(cnt, ctx->counters.p, sizeof(cnt), cudaMemcpyDeviceToHost, s));
    SDD_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    SDD_CUDA(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
    if (stats) {
        stats->steps = cnt[0];
        stats->walks = cnt[1];
        stats->truncated = cnt[2];
        stats->kernel_ms = ms;
        stats->launches = 2;
        stats->items = (int32_t)ni;
        stats->h2d_bytes = ctx->last_h2d + (uint64_t)n_ranges * 2 * sizeof(double) +
                           (node_ids ? (uint64_t)n_ranges * sizeof(uint32_t) : 0);
        stats->d2h_bytes = sb + (uint64_t)n_ranges * sizeof(int64_t) + sizeof(cnt);
    }
    return cnt[2] ? SDD_E_TRUNCATED : SDD_OK;
}

extern "C" sdd_status sdd_range_sums_device(sdd_ctx *ctx, const double *d_nodes_xz, const uint32_t *d_node_ids,
                                            int32_t n_ranges, const int64_t *path_begin,
                                            const int64_t *path_count, double dt, uint64_t seed,
                                            const sdd_config *cfg, double *d_sums, int64_t *d_n_valid,
                                            uint64_t *d_counters, void *stream) {
    sdd_status st = check_ranges(ctx, n_ranges, path_begin, path_count, dt, cfg);
    if (st != SDD_OK) return st;
    if (n_ranges == 0) return SDD_OK;
    if (!d_nodes_xz || !d_sums || !d_n_valid) return fail(SDD_E_ARG, "d_nodes_xz, d_sums and d_n_valid must not be NULL");
    cudaStream_t s = (cudaStream_t)stream;
    st = range_walks(ctx, d_nodes_xz, d_node_ids, n_ranges, path_begin, path_count, dt, seed, cfg, d_sums,
                     reinterpret_cast<long long *>(d_n_valid), s, false, nullptr);
    if (st != SDD_OK) return st;
    if (d_counters)
        SDD_CUDA(cudaMemcpyAsync(d_counters, ctx->counters.p, 3 * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    return SDD_OK;
}

extern "C" sdd_status sdd_reduce_sums_device(sdd_ctx *ctx, int32_t n_nodes, int32_t n_ranges,
                                             const int32_t *range_node, const double *d_sums,
                                             const int64_t *d_n_valid, double *d_mean, double *d_se,
                                             void *stream) {
    if (!ctx) return fail(SDD_E_ARG, "ctx is NULL");
    sdd_status st = range_index(ctx, n_nodes, n_ranges, range_node);
    if (st != SDD_OK) return st;
    if (n_nodes == 0) return SDD_OK;
    if (!d_mean || !d_se || (n_ranges > 0 && (!d_sums || !d_n_valid)))
        return fail(SDD_E_ARG, "d_sums, d_n_valid, d_mean and d_se must not be NULL");
    cudaStream_t s = (cudaStream_t)stream;
    SDD_CUDA(ctx->red_index.ensure(ctx->h_red_index.size() * sizeof(int32_t)));
    SDD_CUDA(cudaMemcpyAsync(ctx->red_index.p, ctx->h_red_index.data(), ctx->h_red_index.size() * sizeof(int32_t),
                             cudaMemcpyHostToDevice, s));
    const int nt = n_nodes * ctx->E;
    range_reduce_kernel<<<(nt + 127) / 128, 128, 0, s>>>(d_sums, reinterpret_cast<const long long *>(d_n_valid),
                                                        (const int32_t *)ctx->red_index.p, n_nodes, ctx->E,
                                                        d_mean, d_se);
    SDD_CUDA(cudaGetLastError());
    return SDD_OK;
}

extern "C" sdd_status sdd_reduce_sums(sdd_ctx *ctx, int32_t n_nodes, int32_t n_ranges, const int32_t *range_node,
                                      const double *sums, const int64_t *n_valid, double *mean, double *se) {
    if (!ctx) return fail(SDD_E_ARG, "ctx is NULL");
    if (n_nodes > 0 && (!mean || !se || (n_ranges > 0 && (!sums || !n_valid))))
        return fail(SDD_E_ARG, "sums, n_valid, mean and se must not be NULL");
    if (n_ranges < 0 || n_nodes <= 0) return sdd_reduce_sums_device(ctx, n_nodes, n_ranges, range_node, nullptr,
                                                                     nullptr, nullptr, nullptr, ctx->stream);
    cudaStream_t s = ctx->stream;
    const size_t sb = (size_t)n_ranges * ctx->E * 4 * sizeof(double);
    const size_t ob = (size_t)n_nodes * ctx->E * 2 * sizeof(double);
    // the walk scratch is free between calls: sums in slots, counts in trunc,
    // outputs in mean / se
    SDD_CUDA(ctx->slots.ensure(std::max<size_t>(sb, 8)));
    SDD_CUDA(ctx->trunc.ensure(std::max<size_t>((size_t)n_ranges * sizeof(int64_t), 8)));
    SDD_CUDA(ctx->mean.ensure(ob));
    SDD_CUDA(ctx->se.ensure(ob));
    if (n_ranges > 0) {
        SDD_CUDA(cudaMemcpyAsync(ctx->slots.p, sums, sb, cudaMemcpyHostToDevice, s));
        SDD_CUDA(cudaMemcpyAsync(ctx->trunc.p, n_valid, (size_t)n_ranges * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    }
    sdd_status st = sdd_reduce_sums_device(ctx, n_nodes, n_ranges, range_node, (const double *)ctx->slots.p,
                                           (const int64_t *)ctx->trunc.p, (double *)ctx->mean.p,
                                           (double *)ctx->se.p, s);
    if (st != SDD_OK) return st;
    SDD_CUDA(cudaMemcpyAsync(mean, ctx->mean.p, ob, cudaMemcpyDeviceToHost, s));
    SDD_CUDA(cudaMemcpyAsync(se, ctx->se.p, ob, cudaMemcpyDeviceToHost, s));
    SDD_CUDA(cudaStreamSynchronize(s));
    return SDD_OK;
}

// ---------------------------------------------------------------------------
// Asynchronous requests (sdd_interface_values_async, sdd_poll, sdd_wait,
// sdd_cancel, sdd_request_result, sdd_request_free).
//
// A request owns its scratch -- one device block (nodes, node ids, item
// table, per-item sums, counters, work queue, outputs) and one page-locked
// host block (the staged inputs and the outputs) -- so several requests of
// one context can be in flight at once, on one stream or several.  Its
// walks are those of sdd_interface_values: the same plan, launch and fixed-
// order reduction, queued on the request's stream.  Cancelling sets the
// request's cancel flag from a side stream: a warp that finds it set when it
// next refills its lanes hands out no more paths, so the launch ends once
// the walks in flight are done.

struct sdd_request {
    sdd_ctx *ctx = nullptr;
    int32_t n_nodes = 0, E = 0;
    size_t n_items = 0;
    cudaStream_t stream = nullptr;  // the caller's, or own_stream
    cudaStream_t own_stream = nullptr, cancel_stream = nullptr;
    cudaEvent_t done = nullptr, ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t armed = nullptr;  // after the memset that clears the cancel flag
    unsigned char *dev = nullptr, *host = nullptr;
    size_t off_mean = 0, off_se = 0, off_cnt = 0, off_flag = 0, off_cancel = 0;
    Launch L{};
    uint64_t h2d = 0;
    std::atomic<int> cancelled{0};
    bool finished = false;
    sdd_status status = SDD_OK;
    std::mutex mu;
};

namespace {

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

void request_release(sdd_request *r) {
    if (r->done) cudaEventSynchronize(r->done);
    if (r->cancel_stream) cudaStreamSynchronize(r->cancel_stream);
    if (r->dev) cudaFree(r->dev);
    if (r->host) cudaFreeHost(r->host);
    if (r->done) cudaEventDestroy(r->done);
    if (r->ev0) cudaEventDestroy(r->ev0);
    if (r->ev1) cudaEventDestroy(r->ev1);
    if (r->armed) cudaEventDestroy(r->armed);
    if (r->own_stream) cudaStreamDestroy(r->own_stream);
    if (r->cancel_stream) cudaStreamDestroy(r->cancel_stream);
    delete r;
}

// Completion of a request whose done event has fired (caller holds r->mu).
void request_finish(sdd_request *r) {
    if (r->finished) return;
    r->finished = true;
    const unsigned long long *cnt = reinterpret_cast<const unsigned long long *>(r->host + r->off_cnt);
    if (r->cancelled.load()) r->status = SDD_E_CANCELLED;
    else r->status = cnt[2] ? SDD_E_TRUNCATED : SDD_OK;
}

}  // namespace

extern "C" sdd_status sdd_interface_values_async(sdd_ctx *ctx, const double *nodes_xz, const uint32_t *node_ids,
                                                 int32_t n_nodes, const int64_t *n_paths, double dt,
                                                 uint64_t seed, const sdd_config *cfg, void *stream,
                                                 sdd_request **out) {
    if (!out) return fail(SDD_E_ARG, "out is NULL");
    *out = nullptr;
    sdd_status st = check_call(ctx, n_nodes, n_paths, dt, cfg);
    if (st != SDD_OK) return st;
    if (n_nodes > 0 && !nodes_xz) return fail(SDD_E_ARG, "nodes_xz is NULL");
    if (cfg && cfg->use_graph) return fail(SDD_E_UNSUPPORTED, "asynchronous requests launch their kernels directly");
    st = check_nodes(ctx, nodes_xz, n_nodes);
    if (st != SDD_OK) return st;
    int device = -1;
    SDD_CUDA(cudaGetDevice(&device));
    if (device != ctx->device) return fail(SDD_E_ARG, "the context's device is not the current device");
    Launch L;
    {
        std::lock_guard<std::mutex> lk(ctx->submit_mu);
        L = choose_launch(ctx, cfg, dt);
    }
    const Plan P = plan_work(n_nodes, nullptr, n_paths, 0, L);
    sdd_request *r = new (std::nothrow) sdd_request();
    if (!r) return fail(SDD_E_OOM, "host allocation failed");
    r->ctx = ctx;
    r->n_nodes = n_nodes;
    r->E = ctx->E;
    r->n_items = P.items.size();
    r->L = L;
    const size_t ni = P.items.size(), nn = (size_t)n_nodes, E = (size_t)ctx->E;
    // one layout for both blocks: inputs (staged on the host, copied once),
    // then device-only scratch, then the outputs (copied back)
    const size_t o_nodes = 0, o_ids = al256(o_nodes + nn * 16), o_items = al256(o_ids + nn * 4);
    const size_t o_i0 = al256(o_items + ni * sizeof(Item)), o_order = al256(o_i0 + (nn + 1) * 4);
    const size_t in_bytes = al256(o_order + P.order.size() * 4);
    const size_t o_slots = in_bytes, o_trunc = al256(o_slots + std::max<size_t>(ni, 1) * E * 32);
    const size_t o_queue = al256(o_trunc + ni * 4), o_err = o_queue + 16, o_flag = o_queue + 24;
    const size_t o_mean = al256(o_err + 16), o_se = al256(o_mean + nn * E * 16), o_cnt = al256(o_se + nn * E * 16);
    const size_t total = al256(o_cnt + 32), o_cancel = total;
    r->off_mean = o_mean; r->off_se = o_se; r->off_cnt = o_cnt; r->off_flag = o_flag; r->off_cancel = o_cancel;
    cudaError_t e = cudaMalloc((void **)&r->dev, total);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&r->host, total + 256);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&r->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&r->ev1);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->armed, cudaEventDisableTiming);
    if (e == cudaSuccess && !stream) e = cudaStreamCreateWithFlags(&r->own_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        request_release(r);
        return e == cudaErrorMemoryAllocation ? fail(SDD_E_OOM, "request allocation") : cuda_fail(e, "request setup");
    }
    r->stream = stream ? (cudaStream_t)stream : r->own_stream;
    unsigned char *h = r->host;
    if (nn) std::memcpy(h + o_nodes, nodes_xz, nn * 16);
    if (node_ids) std::memcpy(h + o_ids, node_ids, nn * 4);
    if (ni) std::memcpy(h + o_items, P.items.data(), ni * sizeof(Item));
    std::memcpy(h + o_i0, P.node_item0.data(), (nn + 1) * 4);
    if (!P.order.empty()) std::memcpy(h + o_order, P.order.data(), P.order.size() * 4);
    *reinterpret_cast<int32_t *>(h + o_cancel) = 1;
    std::memset(h + o_cnt, 0, 32);
    cudaStream_t s = r->stream;
    r->h2d = in_bytes;
    sdd_status res = SDD_OK;
    auto q = [&](cudaError_t err, const char *what) {
        if (err != cudaSuccess && res == SDD_OK) res = cuda_fail(err, what);
    };
    q(cudaMemcpyAsync(r->dev, r->host, in_bytes, cudaMemcpyHostToDevice, s), "request upload");
    if (ni > 0) {
        q(cudaMemsetAsync(r->dev + o_queue, 0, 32, s), "request queue");
        q(cudaMemsetAsync(r->dev + o_cnt, 0, 32, s), "request counters");
        // a cancel copy waits for this point, so the memset cannot clear it
        q(cudaEventRecord(r->armed, s), "event");
        WalkArgs A = base_args(ctx, L, dt, seed);
        A.nodes = reinterpret_cast<const double *>(r->dev + o_nodes);
        A.node_ids = node_ids ? reinterpret_cast<const uint32_t *>(r->dev + o_ids) : nullptr;
        A.items = reinterpret_cast<const Item *>(r->dev + o_items);
        A.n_items = (int32_t)ni;
        A.order = P.order.empty() ? nullptr : reinterpret_cast<const int32_t *>(r->dev + o_order);
        A.slots = reinterpret_cast<double *>(r->dev + o_slots);
        A.item_trunc = reinterpret_cast<int32_t *>(r->dev + o_trunc);
        A.counters = reinterpret_cast<unsigned long long *>(r->dev + o_cnt);
        A.queue = reinterpret_cast<int32_t *>(r->dev + o_queue);
        A.error = reinterpret_cast<int32_t *>(r->dev + o_err);
        A.cancel = reinterpret_cast<const int32_t *>(r->dev + o_flag);
        const int wpc = L.block / 32;
        int grid = L.grid;
        const int need = (int)((ni + wpc - 1) / wpc);
        if (grid > need) grid = need;
        q(cudaEventRecord(r->ev0, s), "event");
        if (res == SDD_OK) {
            cudaError_t le = L.f64 ? launch_walk_f64(L.kmax, ctx->geo, ctx->M, A, grid, L.block, s)
                                   : launch_walk_f32(L.kmax, ctx->geo, ctx->M, A, grid, L.block, s);
            q(le, "walk kernel launch");
        }
        q(cudaEventRecord(r->ev1, s), "event");
        if (res == SDD_OK) {
            const int nt = n_nodes * ctx->E;
            reduce_kernel<<<(nt + 127) / 128, 128, 0, s>>>(
                A.slots, A.item_trunc, A.items, reinterpret_cast<const int32_t *>(r->dev + o_i0), n_nodes, ctx->E,
                reinterpret_cast<double *>(r->dev + o_mean), reinterpret_cast<double *>(r->dev + o_se));
            q(cudaGetLastError(), "reduce kernel launch");
        }
        q(cudaMemcpyAsync(r->host + o_mean, r->dev + o_mean, total - o_mean, cudaMemcpyDeviceToHost, s),
          "request download");
    }
    q(cudaEventRecord(r->done, s), "event");
    if (res != SDD_OK) {
        request_release(r);
        return res;
    }
    *out = r;
    return SDD_OK;
}

extern "C" sdd_status sdd_poll(sdd_request *r) {
    if (!r) return fail(SDD_E_ARG, "request is NULL");
    std::lock_guard<std::mutex> lk(r->mu);
    if (r->finished) return r->status;
    const cudaError_t e = cudaEventQuery(r->done);
    if (e == cudaErrorNotReady) return SDD_E_BUSY;
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventQuery");
    request_finish(r);
    return r->status;
}

extern "C" sdd_status sdd_wait(sdd_request *r, int64_t timeout_ms) {
    if (!r) return fail(SDD_E_ARG, "request is NULL");
    if (timeout_ms < 0) {
        const cudaError_t e = cudaEventSynchronize(r->done);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
        return sdd_poll(r);
    }
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const sdd_status st = sdd_poll(r);
        if (st != SDD_E_BUSY) return st;
        if (std::chrono::steady_clock::now() - t0 >= std::chrono::milliseconds(timeout_ms))
            return SDD_E_TIMEOUT;
        std::this_thread::sleep_for(std::chrono::microseconds(100));
    }
}

extern "C" sdd_status sdd_cancel(sdd_request *r) {
    if (!r) return fail(SDD_E_ARG, "request is NULL");
    std::lock_guard<std::mutex> lk(r->mu);
    if (r->finished || r->cancelled.exchange(1)) return SDD_OK;
    if (r->n_items == 0) return SDD_OK;
    cudaError_t e = cudaSuccess;
    if (!r->cancel_stream) e = cudaStreamCreateWithFlags(&r->cancel_stream, cudaStreamNonBlocking);
    // after the request's queue memset (which also clears the flag), even
    // while the request still waits behind earlier work on its stream
    if (e == cudaSuccess) e = cudaStreamWaitEvent(r->cancel_stream, r->armed, 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(r->dev + r->off_flag, r->host + r->off_cancel, sizeof(int32_t), cudaMemcpyHostToDevice,
                            r->cancel_stream);
    if (e != cudaSuccess) return cuda_fail(e, "cancel");
    return SDD_OK;
}

extern "C" sdd_status sdd_request_result(sdd_request *r, double *mean, double *se, sdd_stats *stats) {
    const sdd_status st = sdd_poll(r);
    if (st != SDD_OK && st != SDD_E_TRUNCATED) return st;
    const size_t ob = (size_t)r->n_nodes * r->E * 16;
    if (r->n_nodes > 0 && (!mean || !se)) return fail(SDD_E_ARG, "mean and se must not be NULL");
    if (ob) {
        std::memcpy(mean, r->host + r->off_mean, ob);
        std::memcpy(se, r->host + r->off_se, ob);
    }
    if (stats) {
        std::memset(stats, 0, sizeof(*stats));
        const unsigned long long *cnt = reinterpret_cast<const unsigned long long *>(r->host + r->off_cnt);
        stats->steps = cnt[0];
        stats->walks = cnt[1];
        stats->truncated = cnt[2];
        float ms = 0.f;
        if (r->n_items && cudaEventElapsedTime(&ms, r->ev0, r->ev1) == cudaSuccess) stats->kernel_ms = ms;
        stats->launches = r->n_items ? 2 : 0;
        stats->items = (int32_t)r->n_items;
        stats->grid = r->L.grid;
        stats->block = r->L.block;
        stats->h2d_bytes = r->h2d;
        stats->d2h_bytes = r->n_items ? r->off_cancel - r->off_mean : 0;
    }
    return st;
}

extern "C" void sdd_request_free(sdd_request *r) {
    if (r) request_release(r);
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
    Launch L = choose_launch(ctx, cfg, dt);
    WalkArgs A = base_args(ctx, L, dt, seed);
    A.nodes = (const double *)ctx->nodes.p;
    if (node_ids) {
        SDD_CUDA(ctx->node_ids.ensure((size_t)n_nodes * sizeof(uint32_t)));
        SDD_CUDA(cudaMemcpyAsync(ctx->node_ids.p, node_ids, (size_t)n_nodes * sizeof(uint32_t),
                                 cudaMemcpyHostToDevice, s));
        A.node_ids = (const uint32_t *)ctx->node_ids.p;
    }
    ctx->plan_valid = false;
    Plan P1 = plan_work(n_nodes, begin.data(), pilot.data(), 0, L);
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
        L = choose_launch(ctx, cfg, dt);
        WalkArgs A2 = base_args(ctx, L, dt, seed);
        A2.nodes = A.nodes;
        A2.node_ids = A.node_ids;
        Plan P2 = plan_work(n_nodes, begin.data(), extra.data(), 0, L);
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

// ---------------------------------------------------------------------------
// Batched launches over several models (sdd_batch_values).

namespace {

sdd_status check_batch(const sdd_batch_entry *en, int32_t n, double dt, const sdd_config *cfg) {
    if (!en || n < 1 || n > kMaxBatchModels) return fail(SDD_E_ARG, "need 1..256 batch entries");
    if (cfg && cfg->precision == SDD_FP64) return fail(SDD_E_UNSUPPORTED, "batched launches run the FP32 walk");
    const sdd_ctx *c0 = en[0].ctx;
    for (int i = 0; i < n; ++i) {
        const sdd_ctx *c = en[i].ctx;
        sdd_status st = check_call(const_cast<sdd_ctx *>(c), en[i].n_nodes, en[i].n_paths, dt, cfg);
        if (st != SDD_OK) return st;
        if (c->geo != GEO_RASTER) return fail(SDD_E_UNSUPPORTED, "batched launches need raster models");
        if (c->M.nx != c0->M.nx || c->M.nz != c0->M.nz || c->M.xmin != c0->M.xmin ||
            c->M.xmax != c0->M.xmax || c->M.zmin != c0->M.zmin || c->M.zmax != c0->M.zmax ||
            c->E != c0->E || c->M.g_kind != c0->M.g_kind || c->device != c0->device)
            return fail(SDD_E_ARG, "batched models must share device, domain, raster size, n_eval and g_kind");
        if (en[i].n_nodes > 0 && (!en[i].nodes_xz || !en[i].mean || !en[i].se))
            return fail(SDD_E_ARG, "entry nodes_xz, mean and se must not be NULL");
        st = check_nodes(c, en[i].nodes_xz, en[i].n_nodes);
        if (st != SDD_OK) return st;
    }
    return SDD_OK;
}

}  // namespace

extern "C" sdd_status sdd_batch_values(const sdd_batch_entry *entries, int32_t n_entries, double dt,
                                       uint64_t seed, const sdd_config *cfg, sdd_stats *stats) {
    sdd_status st = check_batch(entries, n_entries, dt, cfg);
    if (st != SDD_OK) return st;
    if (stats) std::memset(stats, 0, sizeof(*stats));
    sdd_ctx *own = entries[0].ctx;
    // concatenated nodes, ids and path counts; model index per node
    std::vector<double> nodes;
    std::vector<uint32_t> ids;
    std::vector<int64_t> paths;
    std::vector<int32_t> node_model, first(n_entries + 1);
    int Kmax = 1;
    for (int i = 0; i < n_entries; ++i) {
        const sdd_batch_entry &e = entries[i];
        first[i] = (int32_t)paths.size();
        for (int j = 0; j < e.n_nodes; ++j) {
            nodes.push_back(e.nodes_xz[2 * j]);
            nodes.push_back(e.nodes_xz[2 * j + 1]);
            ids.push_back(e.node_ids ? e.node_ids[j] : (uint32_t)j);
            paths.push_back(e.n_paths[j]);
            node_model.push_back(i);
        }
        Kmax = std::max(Kmax, e.ctx->K);
    }
    const int32_t n_nodes = (int32_t)paths.size();
    first[n_entries] = n_nodes;
    if (n_nodes == 0) return SDD_OK;
    const Launch L = choose_launch(own, cfg, dt, kmax_for(Kmax), GC_RASTER_MULTI);
    Plan P = L.chunk > 0 ? plan_work(n_nodes, nullptr, paths.data(), 0, L)
                         : plan_grouped(n_nodes, nullptr, paths.data(), node_model.data(), n_entries, L);
    for (Item &I : P.items) I.model = node_model[I.node];
    own->plan_valid = false;

    std::vector<BatchModel> table(n_entries);
    for (int i = 0; i < n_entries; ++i) {
        const sdd_ctx *c = entries[i].ctx;
        BatchModel &B = table[i];
        std::memset(&B, 0, sizeof(B));
        B.raster = c->M.raster;
        B.tcoarse = c->M.tcoarse;
        B.tpool = c->M.tpool;
        B.K = c->K;
        for (int k = 0; k < c->E * c->K; ++k) B.kappa[k] = c->M.kappa[k];
        for (int k = 0; k < c->E; ++k) B.ev[k] = c->M.ev[k];
    }
    cudaStream_t s = own->stream;
    const size_t ob = (size_t)n_nodes * own->E * 2 * sizeof(double);
    SDD_CUDA(own->batch_models.ensure(table.size() * sizeof(BatchModel)));
    SDD_CUDA(own->nodes.ensure(nodes.size() * sizeof(double)));
    SDD_CUDA(own->node_ids.ensure(ids.size() * sizeof(uint32_t)));
    SDD_CUDA(own->mean.ensure(ob));
    SDD_CUDA(own->se.ensure(ob));
    SDD_CUDA(cudaMemcpyAsync(own->batch_models.p, table.data(), table.size() * sizeof(BatchModel),
                             cudaMemcpyHostToDevice, s));
    SDD_CUDA(cudaMemcpyAsync(own->nodes.p, nodes.data(), nodes.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    SDD_CUDA(cudaMemcpyAsync(own->node_ids.p, ids.data(), ids.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    ModelDev Mb = own->M;
    Mb.gcode = GC_RASTER_MULTI;
    Mb.K = Kmax;
    WalkArgs A = base_args(own, L, dt, seed);
    A.nodes = (const double *)own->nodes.p;
    A.node_ids = (const uint32_t *)own->node_ids.p;
    A.models = (const BatchModel *)own->batch_models.p;
    st = run(own, P, L, A, s, true, true, (double *)own->mean.p, (double *)own->se.p, n_nodes, &Mb);
    if (st != SDD_OK) return st;
    std::vector<double> hm(ob / sizeof(double)), hs(ob / sizeof(double));
    unsigned long long cnt[3] = {0, 0, 0};
    SDD_CUDA(cudaMemcpyAsync(hm.data(), own->mean.p, ob, cudaMemcpyDeviceToHost, s));
    SDD_CUDA(cudaMemcpyAsync(hs.data(), own->se.p, ob, cudaMemcpyDeviceToHost, s));
    SDD_CUDA(cudaMemcpyAsync(cnt, own->counters.p, sizeof(cnt), cudaMemcpyDeviceToHost, s));
    SDD_CUDA(cudaStreamSynchronize(s));
    const size_t per = (size_t)own->E * 2;
    for (int i = 0; i < n_entries; ++i) {
        const size_t o = (size_t)first[i] * per, nb = (size_t)(first[i + 1] - first[i]) * per;
        if (nb == 0) continue;
        std::memcpy(entries[i].mean, hm.data() + o, nb * sizeof(double));
        std::memcpy(entries[i].se, hs.data() + o, nb * sizeof(double));
    }
    if (stats) {
        float ms = 0.f;
        SDD_CUDA(cudaEventElapsedTime(&ms, own->ev0, own->ev1));
        stats->steps = cnt[0];
        stats->walks = cnt[1];
        stats->truncated = cnt[2];
        stats->kernel_ms = ms;
        stats->launches = 2;
        stats->items = (int32_t)P.items.size();
        stats->grid = L.grid;
        stats->block = L.block;
        stats->h2d_bytes = table.size() * sizeof(BatchModel) + nodes.size() * 8 + ids.size() * 4 +
                           P.items.size() * sizeof(Item);
        stats->d2h_bytes = 2 * ob + sizeof(cnt);
    }
    return cnt[2] ? SDD_E_TRUNCATED : SDD_OK;
}

// ---------------------------------------------------------------------------
// Serving (sdd_server_*): admission, continuous batching, completion.

namespace {

using Clock = std::chrono::steady_clock;

double us_since(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::micro>(b - a).count();
}

struct SrvRequest {
    uint64_t id = 0;
    int slot = -1;                 // arena slot (tile map)
    int64_t bytes = 0;
    BatchModel bm;                 // tile map, rates and boundary constants
    int K = 1;
    std::vector<double> nodes;
    std::vector<uint32_t> ids;
    std::vector<int64_t> fixed;    // fixed counts, empty when adaptive
    double target_se = 0.0;
    int64_t n_pilot = 0, n_max = 0;
    int phase = 0;                 // 0 first walks, 2 top-up walks, 4 finished
    int pieces_left = 0;           // pieces of the current phase not yet folded in
    std::vector<int64_t> begin, count;
    std::vector<double> sums;      // [n][E][4]
    std::vector<long long> nvalid;
    std::vector<int64_t> n_used;
    bool cancelled = false;
    sdd_status status = SDD_OK;
    uint64_t walks = 0, truncated = 0;
    int launches = 0;
    Clock::time_point t_submit, t_first, t_done;
    bool started = false;
    double deadline = 0.0;         // queue key of the current phase (seconds, virtual)
};

// Nodes [a, b) of a request's current phase, launched together.
struct SrvPiece {
    SrvRequest *r;
    int32_t a, b;
    int64_t walks;
};

struct SrvPart {
    SrvRequest *r;
    int32_t node0;  // first node of the piece in the launch's node list
    int32_t a, b;   // the piece's nodes in the request
};

struct SrvLane {
    cudaStream_t s = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool busy = false;
    DevBuf items, slots, trunc, counters, queue, err, nodes, ids, models, sums, nvalid;
    double *h_sums = nullptr;
    long long *h_nvalid = nullptr;
    unsigned long long *h_cnt = nullptr;
    size_t h_cap_nodes = 0;
    std::vector<SrvPart> parts;
    int32_t n_nodes = 0;
    uint64_t walks = 0;
};

}  // namespace

struct sdd_server {
    sdd_server_config cfg;
    int device = 0;
    sdd_ctx *tmpl = nullptr;       // a context with the server's model shape (launch planning)
    DevBuf arena;                  // max_requests tile maps of slot_bytes each
    size_t coarse_bytes = 0, slot_bytes = 0;
    std::vector<int> free_slots;
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::map<uint64_t, SrvRequest *> reqs;
    std::deque<SrvPiece> runnable;
    int64_t batch_walks = 0;       // walk budget of one launch
    std::vector<SrvLane> lanes;
    std::thread worker;
    bool stop = false;
    uint64_t next_id = 1;
    int64_t bytes_in_use = 0;
    sdd_server_stats st{};
    std::string worker_error;
    Clock::time_point t_start = Clock::now();  // origin of the virtual deadlines
};

namespace {

int64_t request_bytes(const sdd_server *srv, int32_t n_nodes) {
    const int E = srv->cfg.n_eval;
    return (int64_t)srv->slot_bytes + (int64_t)n_nodes * (16 + 4 + 8 + 8 + 32 * E) +
           (int64_t)sizeof(BatchModel);
}

// Walks a launch gets through per second, for the virtual deadlines below
// (a scale only: the order of the queue depends on it, not the results), and
// the most a phase's own walk time adds to its deadline: a large request can
// only be overtaken by requests submitted less than that after it.
constexpr double kDeadlineWalksPerS = 5.0e8;
constexpr double kDeadlineCapS = 1.0;

// Cut a request's current phase into pieces of at most batch_walks walks
// (whole nodes; nodes with no walks left out) and queue them by the phase's
// virtual deadline: the request's submission time plus the time its phase's
// walks would take alone, at most kDeadlineCapS.  A small request (or a pilot phase) then goes ahead
// of a large top-up submitted a little earlier, while a request submitted
// long before keeps its place; every deadline grows with the submission
// time, so no request waits forever.  Launches serve the earliest deadline
// and fill up with the next ones.
void srv_queue_phase(sdd_server *srv, SrvRequest *r, Clock::time_point t0) {
    const int32_t n = (int32_t)r->ids.size();
    int pieces = 0;
    long long phase_walks = 0;
    for (int32_t j = 0; j < n; ++j) phase_walks += r->count[j];
    r->deadline = std::chrono::duration<double>(r->t_submit - t0).count() +
                  std::min((double)phase_walks / kDeadlineWalksPerS, kDeadlineCapS);
    auto at = std::upper_bound(srv->runnable.begin(), srv->runnable.end(), r->deadline,
                               [](double d, const SrvPiece &pc) { return d < pc.r->deadline; });
    std::vector<SrvPiece> add;
    int32_t a = 0;
    while (a < n) {
        while (a < n && r->count[a] == 0) ++a;
        if (a >= n) break;
        int32_t b = a;
        int64_t w = 0;
        while (b < n && (b == a || w + r->count[b] <= srv->batch_walks)) {
            w += r->count[b];
            ++b;
            while (b < n && r->count[b] == 0) ++b;
        }
        add.push_back({r, a, b, w});
        ++pieces;
        a = b;
    }
    srv->runnable.insert(at, add.begin(), add.end());
    r->pieces_left = pieces;
}

// Queue one launch over the pieces: each piece's nodes with their current
// ranges, one model-table entry per request.
sdd_status srv_launch(sdd_server *srv, SrvLane &L, std::vector<SrvPiece> &batch) {
    const int E = srv->cfg.n_eval;
    std::vector<double> nodes;
    std::vector<uint32_t> ids;
    std::vector<int64_t> begin, count;
    std::vector<int32_t> node_model;
    std::vector<BatchModel> table;
    std::map<SrvRequest *, int32_t> model_of;
    L.parts.clear();
    int Kmax = 1;
    for (const SrvPiece &pc : batch) {
        SrvRequest *r = pc.r;
        auto it = model_of.find(r);
        int32_t m;
        if (it == model_of.end()) {
            m = (int32_t)table.size();
            model_of[r] = m;
            table.push_back(r->bm);
            Kmax = std::max(Kmax, r->K);
        } else {
            m = it->second;
        }
        L.parts.push_back({r, (int32_t)ids.size(), pc.a, pc.b});
        for (int j = pc.a; j < pc.b; ++j) {
            nodes.push_back(r->nodes[2 * j]);
            nodes.push_back(r->nodes[2 * j + 1]);
            ids.push_back(r->ids[j]);
            begin.push_back(r->begin[j]);
            count.push_back(r->count[j]);
            node_model.push_back(m);
        }
    }
    const int32_t n_nodes = (int32_t)ids.size();
    L.n_nodes = n_nodes;
    long long total = 0;
    for (int64_t c : count) total += c;
    L.walks = (uint64_t)total;
    const Launch La = choose_launch(srv->tmpl, &srv->cfg.launch, srv->cfg.dt, kmax_for(Kmax),
                                    GC_RASTER_MULTI);
    Plan P = La.chunk > 0 ? plan_work(n_nodes, begin.data(), count.data(), 0, La)
                          : plan_grouped(n_nodes, begin.data(), count.data(), node_model.data(),
                                         (int32_t)table.size(), La);
    for (Item &I : P.items) I.model = node_model[I.node];
    const size_t ni = P.items.size();
    cudaStream_t s = L.s;
    const size_t tb = table_bytes(P, n_nodes);
    SDD_CUDA(L.items.ensure(tb));
    SDD_CUDA(L.slots.ensure(std::max<size_t>(ni, 1) * (size_t)E * 4 * sizeof(double)));
    SDD_CUDA(L.trunc.ensure(std::max<size_t>(ni, 1) * sizeof(int32_t)));
    SDD_CUDA(L.counters.ensure(3 * sizeof(unsigned long long)));
    SDD_CUDA(L.queue.ensure(std::max<size_t>(P.qbase.size(), 1) * sizeof(int32_t)));
    SDD_CUDA(L.err.ensure(sizeof(int32_t)));
    SDD_CUDA(L.nodes.ensure(nodes.size() * sizeof(double)));
    SDD_CUDA(L.ids.ensure(ids.size() * sizeof(uint32_t)));
    SDD_CUDA(L.models.ensure(table.size() * sizeof(BatchModel)));
    SDD_CUDA(L.sums.ensure((size_t)n_nodes * E * 4 * sizeof(double)));
    SDD_CUDA(L.nvalid.ensure((size_t)n_nodes * sizeof(long long)));
    if ((size_t)n_nodes > L.h_cap_nodes) {
        if (L.h_sums) cudaFreeHost(L.h_sums);
        if (L.h_nvalid) cudaFreeHost(L.h_nvalid);
        L.h_sums = nullptr;
        L.h_nvalid = nullptr;
        L.h_cap_nodes = 0;
        SDD_CUDA(cudaMallocHost((void **)&L.h_sums, (size_t)n_nodes * E * 4 * sizeof(double)));
        SDD_CUDA(cudaMallocHost((void **)&L.h_nvalid, (size_t)n_nodes * sizeof(long long)));
        L.h_cap_nodes = n_nodes;
    }
    std::vector<unsigned char> hi(tb);
    pack_table(P, n_nodes, hi.data());
    SDD_CUDA(cudaMemcpyAsync(L.items.p, hi.data(), hi.size(), cudaMemcpyHostToDevice, s));
    SDD_CUDA(cudaMemcpyAsync(L.nodes.p, nodes.data(), nodes.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    SDD_CUDA(cudaMemcpyAsync(L.ids.p, ids.data(), ids.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    SDD_CUDA(cudaMemcpyAsync(L.models.p, table.data(), table.size() * sizeof(BatchModel), cudaMemcpyHostToDevice, s));
    SDD_CUDA(cudaMemsetAsync(L.queue.p, 0, std::max<size_t>(P.qbase.size(), 1) * sizeof(int32_t), s));
    SDD_CUDA(cudaMemsetAsync(L.counters.p, 0, 3 * sizeof(unsigned long long), s));
    WalkArgs A = base_args(srv->tmpl, La, srv->cfg.dt, srv->cfg.seed);
    A.items = (const Item *)L.items.p;
    A.n_items = (int32_t)ni;
    table_args(P, n_nodes, reinterpret_cast<const unsigned char *>(L.items.p), A);
    A.nodes = (const double *)L.nodes.p;
    A.node_ids = (const uint32_t *)L.ids.p;
    A.slots = (double *)L.slots.p;
    A.item_trunc = (int32_t *)L.trunc.p;
    A.counters = (unsigned long long *)L.counters.p;
    A.queue = (int32_t *)L.queue.p;
    A.error = (int32_t *)L.err.p;
    A.models = (const BatchModel *)L.models.p;
    ModelDev Mb = srv->tmpl->M;
    Mb.gcode = GC_RASTER_MULTI;
    Mb.K = Kmax;
    const int wpc = La.block / 32;
    int grid = La.grid;
    const int need = (int)((ni + wpc - 1) / wpc);
    if (grid > need) grid = need;
    SDD_CUDA(cudaEventRecord(L.ev0, s));
    if (ni > 0) {
        cudaError_t e = launch_walk_f32(La.kmax, GEO_RASTER, Mb, A, grid, La.block, s);
        if (e != cudaSuccess) return cuda_fail(e, "batched walk launch");
    }
    SDD_CUDA(cudaEventRecord(L.ev1, s));
    const int nt = n_nodes * E;
    sums_kernel<<<(nt + 127) / 128, 128, 0, s>>>(A.slots, A.item_trunc, A.items,
                                                reinterpret_cast<const int32_t *>((const unsigned char *)L.items.p + ni * sizeof(Item)),
                                                n_nodes, E, (double *)L.sums.p, (long long *)L.nvalid.p);
    SDD_CUDA(cudaGetLastError());
    SDD_CUDA(cudaMemcpyAsync(L.h_sums, L.sums.p, (size_t)n_nodes * E * 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    SDD_CUDA(cudaMemcpyAsync(L.h_nvalid, L.nvalid.p, (size_t)n_nodes * sizeof(long long), cudaMemcpyDeviceToHost, s));
    SDD_CUDA(cudaMemcpyAsync(L.h_cnt, L.counters.p, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    L.busy = true;
    return SDD_OK;
}

// A request ends: its status and the counters.
void srv_finish(sdd_server *srv, SrvRequest *r) {
    r->phase = 4;
    r->t_done = Clock::now();
    if (r->cancelled) r->status = SDD_E_CANCELLED;
    else if (r->status == SDD_OK && r->truncated) r->status = SDD_E_TRUNCATED;
    srv->st.completed += 1;
    if (r->cancelled) srv->st.cancelled += 1;
}

// All pieces of a request's phase are in: size the top-up from the pilot,
// or finish.
void srv_phase_done(sdd_server *srv, SrvRequest *r) {
    const int E = srv->cfg.n_eval;
    if (r->cancelled) {
        srv_finish(srv, r);
        return;
    }
    if (r->phase == 0 && r->fixed.empty()) {
        const int32_t n = (int32_t)r->ids.size();
        long long extra_total = 0;
        for (int j = 0; j < n; ++j) {
            double need = 0.0;
            for (int e = 0; e < E; ++e) {
                double m[2], sd[2];
                finish(&r->sums[((size_t)j * E + e) * 4], r->nvalid[j], m, sd);
                const double var = (sd[0] * sd[0] + sd[1] * sd[1]) * (double)r->nvalid[j];
                if (std::isfinite(var)) need = std::max(need, var);
            }
            double N = std::ceil(need / (r->target_se * r->target_se));
            if (!(N >= (double)r->n_pilot)) N = (double)r->n_pilot;
            if (N > (double)r->n_max) N = (double)r->n_max;
            r->n_used[j] = (int64_t)N;
            r->begin[j] = r->n_pilot;
            r->count[j] = (int64_t)N - r->n_pilot;
            extra_total += r->count[j];
        }
        if (extra_total > 0) {
            r->phase = 2;
            srv_queue_phase(srv, r, srv->t_start);
            return;
        }
    }
    srv_finish(srv, r);
}

// A launch ended: fold its per-node sums into its requests (the pieces of a
// phase cover disjoint nodes, so the order of their launches does not matter).
void srv_complete(sdd_server *srv, SrvLane &L) {
    const int E = srv->cfg.n_eval;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, L.ev0, L.ev1);
    srv->st.gpu_busy_ms += ms;
    srv->st.launches += 1;
    srv->st.steps += L.h_cnt[0];
    srv->st.walks += L.h_cnt[1];
    std::map<SrvRequest *, int> seen;
    for (const SrvPart &pt : L.parts) {
        SrvRequest *r = pt.r;
        if (seen[r]++ == 0) r->launches += 1;
        for (int j = pt.a; j < pt.b; ++j) {
            const int32_t k = pt.node0 + (j - pt.a);
            const long long nv = L.h_nvalid[k];
            r->walks += (uint64_t)r->count[j];
            r->truncated += (uint64_t)(r->count[j] - nv);
            r->nvalid[j] += nv;
            for (int q = 0; q < E * 4; ++q)
                r->sums[(size_t)j * E * 4 + q] += L.h_sums[(size_t)k * E * 4 + q];
        }
        if (--r->pieces_left == 0) srv_phase_done(srv, r);
    }
    L.parts.clear();
    L.busy = false;
}

void srv_worker(sdd_server *srv) {
    cudaSetDevice(srv->device);
    std::unique_lock<std::mutex> lk(srv->mu);
    while (true) {
        bool progress = false;
        for (SrvLane &L : srv->lanes) {
            if (L.busy && cudaEventQuery(L.ev1) == cudaSuccess && cudaStreamQuery(L.s) == cudaSuccess) {
                srv_complete(srv, L);
                progress = true;
            }
        }
        if (progress) srv->done_cv.notify_all();
        if (srv->stop) {
            bool any_busy = false;
            for (SrvLane &L : srv->lanes) any_busy |= L.busy;
            if (!any_busy) break;
        }
        for (SrvLane &L : srv->lanes) {
            if (L.busy || srv->runnable.empty() || srv->stop) continue;
            // The launch serves the oldest runnable piece and fills up with the
            // pieces, in queue order, whose models need the same material bound
            // (kmax_for(K): 2, 3, 4 or 8): a batch runs the kernel of its class,
            // so requests with few materials keep the faster per-step counters
            // instead of the shared-memory histogram that one 8-material model
            // would impose on the whole launch.
            std::vector<SrvPiece> batch;
            std::map<SrvRequest *, int> models;
            int64_t walks = 0;
            int cls = 0;
            for (auto it = srv->runnable.begin(); it != srv->runnable.end();) {
                const SrvPiece pc = *it;
                if (pc.r->cancelled) {
                    it = srv->runnable.erase(it);
                    if (--pc.r->pieces_left == 0) srv_finish(srv, pc.r);
                    progress = true;
                    continue;
                }
                const int c = kmax_for(pc.r->K);
                if (batch.empty()) cls = c;
                if (c != cls) {
                    ++it;
                    continue;
                }
                const bool new_model = models.find(pc.r) == models.end();
                if (!batch.empty() && (walks + pc.walks > srv->batch_walks ||
                                       (new_model && (int)models.size() >= srv->cfg.max_batch_models)))
                    break;
                it = srv->runnable.erase(it);
                models[pc.r] = 1;
                walks += pc.walks;
                if (!pc.r->started) {
                    pc.r->started = true;
                    pc.r->t_first = Clock::now();
                }
                batch.push_back(pc);
            }
            if (batch.empty()) continue;
            sdd_status st = srv_launch(srv, L, batch);
            if (st != SDD_OK) {
                srv->worker_error = g_last_error;
                for (const SrvPiece &pc : batch) {
                    pc.r->status = st;
                    pc.r->cancelled = true;
                    if (--pc.r->pieces_left == 0) srv_finish(srv, pc.r);
                }
                L.busy = false;
            }
            progress = true;
        }
        if (progress) {
            srv->done_cv.notify_all();
            continue;
        }
        srv->cv.wait_for(lk, std::chrono::microseconds(50));
    }
}

}  // namespace

extern "C" sdd_status sdd_server_create(const sdd_server_config *cfg, sdd_server **out) {
    if (!out) return fail(SDD_E_ARG, "out is NULL");
    *out = nullptr;
    if (!cfg) return fail(SDD_E_ARG, "cfg is NULL");
    if (cfg->nx < 1 || cfg->nz < 1 || cfg->nx > kMaxRasterSide || cfg->nz > kMaxRasterSide ||
        (long long)cfg->nx * cfg->nz > (1ll << 31))
        return fail(SDD_E_ARG, "raster size out of range");
    if (cfg->n_eval < 1 || cfg->n_eval > SDD_MAX_EVAL) return fail(SDD_E_ARG, "n_eval must be in 1..32");
    if (cfg->max_requests < 1 || cfg->max_requests > 4096) return fail(SDD_E_ARG, "max_requests must be in 1..4096");
    if (cfg->n_streams < 1 || cfg->n_streams > 8) return fail(SDD_E_ARG, "n_streams must be in 1..8");
    if (cfg->max_batch_models < 1 || cfg->max_batch_models > kMaxBatchModels)
        return fail(SDD_E_ARG, "max_batch_models must be in 1..256");
    if (cfg->max_bytes < 0) return fail(SDD_E_ARG, "max_bytes < 0");
    if (cfg->max_batch_walks < 0) return fail(SDD_E_ARG, "max_batch_walks < 0");
    if (cfg->launch.precision != SDD_FP32) return fail(SDD_E_UNSUPPORTED, "the server runs the FP32 walk");
    sdd_status st;
    // a template model of the server's shape (one material, blank raster)
    std::vector<int8_t> blank((size_t)cfg->nx * cfg->nz, 0);
    std::vector<double> kap((size_t)cfg->n_eval, 0.0);
    sdd_model_desc md;
    std::memset(&md, 0, sizeof(md));
    md.domain = cfg->domain;
    md.n_materials = 1;
    md.n_eval = cfg->n_eval;
    md.kappa = kap.data();
    md.raster = blank.data();
    md.nx = cfg->nx;
    md.nz = cfg->nz;
    md.g_kind = cfg->g_kind;
    sdd_server *srv = new (std::nothrow) sdd_server();
    if (!srv) return fail(SDD_E_OOM, "host allocation failed");
    srv->cfg = *cfg;
    srv->batch_walks = cfg->max_batch_walks > 0 ? cfg->max_batch_walks : (int64_t)1 << 24;
    st = sdd_create(&md, &srv->tmpl);
    if (st != SDD_OK) {
        delete srv;
        return st;
    }
    const int64_t np1 = 1;
    st = check_call(srv->tmpl, 1, &np1, cfg->dt, &cfg->launch);
    if (st != SDD_OK) {
        sdd_server_destroy(srv);
        return st;
    }
    srv->device = srv->tmpl->device;
    const size_t ntx = tile_cols(cfg->nx), ntz = tile_cols(cfg->nz);
    srv->coarse_bytes = (ntx * ntz * sizeof(uint32_t) + 255) / 256 * 256;
    srv->slot_bytes = srv->coarse_bytes + ntx * ntz * kTile * kTile;  // pool of every tile mixed at most
    cudaError_t e = srv->arena.ensure((size_t)cfg->max_requests * srv->slot_bytes);
    if (e != cudaSuccess) {
        sdd_server_destroy(srv);
        return fail(SDD_E_OOM, "raster arena allocation failed");
    }
    for (int i = cfg->max_requests - 1; i >= 0; --i) srv->free_slots.push_back(i);
    srv->lanes.resize(cfg->n_streams);
    for (SrvLane &L : srv->lanes) {
        e = cudaStreamCreateWithFlags(&L.s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreate(&L.ev0);
        if (e == cudaSuccess) e = cudaEventCreate(&L.ev1);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&L.h_cnt, 3 * sizeof(unsigned long long));
        if (e != cudaSuccess) {
            sdd_server_destroy(srv);
            return cuda_fail(e, "server stream setup");
        }
    }
    srv->worker = std::thread(srv_worker, srv);
    *out = srv;
    return SDD_OK;
}

extern "C" void sdd_server_destroy(sdd_server *srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv.notify_all();
    if (srv->worker.joinable()) srv->worker.join();
    for (SrvLane &L : srv->lanes) {
        if (L.s) cudaStreamSynchronize(L.s);
        DevBuf *b[] = {&L.items, &L.slots, &L.trunc, &L.counters, &L.queue, &L.err, &L.nodes,
                       &L.ids, &L.models, &L.sums, &L.nvalid};
        for (DevBuf *x : b) x->release();
        if (L.h_sums) cudaFreeHost(L.h_sums);
        if (L.h_nvalid) cudaFreeHost(L.h_nvalid);
        if (L.h_cnt) cudaFreeHost(L.h_cnt);
        if (L.ev0) cudaEventDestroy(L.ev0);
        if (L.ev1) cudaEventDestroy(L.ev1);
        if (L.s) cudaStreamDestroy(L.s);
    }
    for (auto &kv : srv->reqs) delete kv.second;
    srv->arena.release();
    sdd_destroy(srv->tmpl);
    delete srv;
}

extern "C" sdd_status sdd_server_submit(sdd_server *srv, const sdd_request_desc *req, uint64_t *id) {
    if (!srv || !req || !id) return fail(SDD_E_ARG, "srv, req and id must not be NULL");
    const sdd_model_desc *m = req->model;
    sdd_status st = check_model(m);
    if (st != SDD_OK) return st;
    const sdd_server_config &c = srv->cfg;
    if (!m->raster || m->nx != c.nx || m->nz != c.nz || m->n_eval != c.n_eval || m->g_kind != c.g_kind ||
        m->domain.x_min != c.domain.x_min || m->domain.x_max != c.domain.x_max ||
        m->domain.z_min != c.domain.z_min || m->domain.z_max != c.domain.z_max)
        return fail(SDD_E_ARG, "request model does not match the server (raster, size, n_eval, g_kind, domain)");
    if (req->n_nodes < 1 || req->n_nodes > 65536 || !req->nodes_xz)
        return fail(SDD_E_ARG, "n_nodes must be in 1..65536 with nodes_xz");
    if (req->n_paths) {
        for (int j = 0; j < req->n_nodes; ++j)
            if (req->n_paths[j] < 1 || req->n_paths[j] > 0x7fffffffll)
                return fail(SDD_E_ARG, "n_paths must be in 1..2^31-1");
    } else if (!(req->target_se > 0.0) || req->n_pilot < 2 || req->n_max < req->n_pilot ||
               req->n_max > 0x7fffffffll) {
        return fail(SDD_E_ARG, "adaptive requests need target_se > 0 and 2 <= n_pilot <= n_max <= 2^31-1");
    }
    st = check_nodes(srv->tmpl, req->nodes_xz, req->n_nodes);
    if (st != SDD_OK) return st;
    SrvRequest *r = new (std::nothrow) SrvRequest();
    if (!r) return fail(SDD_E_OOM, "host allocation failed");
    ModelDev md;
    build_model(m, md);
    std::memset(&r->bm, 0, sizeof(r->bm));
    r->K = m->n_materials;
    r->bm.K = m->n_materials;
    for (int k = 0; k < md.E * md.K; ++k) r->bm.kappa[k] = md.kappa[k];
    for (int k = 0; k < md.E; ++k) r->bm.ev[k] = md.ev[k];
    const int n = req->n_nodes, E = c.n_eval;
    r->nodes.assign(req->nodes_xz, req->nodes_xz + 2 * n);
    r->ids.resize(n);
    for (int j = 0; j < n; ++j) r->ids[j] = req->node_ids ? req->node_ids[j] : (uint32_t)j;
    r->begin.assign(n, 0);
    r->count.resize(n);
    r->n_used.resize(n);
    if (req->n_paths) {
        r->fixed.assign(req->n_paths, req->n_paths + n);
        for (int j = 0; j < n; ++j) r->count[j] = r->n_used[j] = req->n_paths[j];
    } else {
        r->target_se = req->target_se;
        r->n_pilot = req->n_pilot;
        r->n_max = req->n_max;
        for (int j = 0; j < n; ++j) r->count[j] = r->n_used[j] = req->n_pilot;
    }
    r->sums.assign((size_t)n * E * 4, 0.0);
    r->nvalid.assign(n, 0);
    r->bytes = request_bytes(srv, n);
    std::unique_lock<std::mutex> lk(srv->mu);
    srv->st.submitted += 1;
    if (srv->free_slots.empty() || (c.max_bytes > 0 && srv->bytes_in_use + r->bytes > c.max_bytes)) {
        srv->st.refused += 1;
        lk.unlock();
        delete r;
        return fail(SDD_E_BUSY, "no free slot or device memory; retry later");
    }
    r->slot = srv->free_slots.back();
    srv->free_slots.pop_back();
    srv->bytes_in_use += r->bytes;
    lk.unlock();
    // the slot is reserved: build and upload the tile map without holding the lock
    std::vector<uint32_t> coarse;
    std::vector<uint8_t> pool;
    build_tiles(m->raster, c.nx, c.nz, coarse, pool);
    unsigned char *base = (unsigned char *)srv->arena.p + (size_t)r->slot * srv->slot_bytes;
    r->bm.raster = nullptr;
    r->bm.tcoarse = (const uint32_t *)base;
    r->bm.tpool = base + srv->coarse_bytes;
    int prev = -1;
    cudaError_t e = cudaGetDevice(&prev);
    if (e == cudaSuccess && prev != srv->device) e = cudaSetDevice(srv->device);
    if (e == cudaSuccess)
        e = cudaMemcpy(base, coarse.data(), coarse.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !pool.empty())
        e = cudaMemcpy(base + srv->coarse_bytes, pool.data(), pool.size(), cudaMemcpyHostToDevice);
    if (prev >= 0 && prev != srv->device) cudaSetDevice(prev);
    lk.lock();
    if (e != cudaSuccess) {
        srv->free_slots.push_back(r->slot);
        srv->bytes_in_use -= r->bytes;
        lk.unlock();
        delete r;
        return cuda_fail(e, "raster upload");
    }
    r->id = srv->next_id++;
    r->t_submit = Clock::now();
    srv->reqs[r->id] = r;
    r->phase = 0;
    srv_queue_phase(srv, r, srv->t_start);
    *id = r->id;
    lk.unlock();
    srv->cv.notify_all();
    return SDD_OK;
}

extern "C" sdd_status sdd_server_poll(sdd_server *srv, uint64_t id, int32_t *done) {
    if (!srv || !done) return fail(SDD_E_ARG, "srv and done must not be NULL");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(id);
    if (it == srv->reqs.end()) return fail(SDD_E_ARG, "unknown request id");
    *done = it->second->phase == 4 ? 1 : 0;
    return SDD_OK;
}

extern "C" sdd_status sdd_server_wait(sdd_server *srv, uint64_t id, int64_t timeout_ms) {
    if (!srv) return fail(SDD_E_ARG, "srv is NULL");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(id);
    if (it == srv->reqs.end()) return fail(SDD_E_ARG, "unknown request id");
    SrvRequest *r = it->second;
    auto pred = [&] { return r->phase == 4; };
    if (timeout_ms < 0) {
        srv->done_cv.wait(lk, pred);
        return SDD_OK;
    }
    if (!srv->done_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred))
        return fail(SDD_E_TIMEOUT, "request not finished within the timeout");
    return SDD_OK;
}

extern "C" sdd_status sdd_server_result(sdd_server *srv, uint64_t id, double *mean, double *se,
                                        int64_t *n_used, sdd_request_stats *stats) {
    if (!srv) return fail(SDD_E_ARG, "srv is NULL");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(id);
    if (it == srv->reqs.end()) return fail(SDD_E_ARG, "unknown request id");
    SrvRequest *r = it->second;
    if (r->phase != 4) return fail(SDD_E_BUSY, "request not finished");
    const int E = srv->cfg.n_eval;
    const int n = (int)r->ids.size();
    if (r->status == SDD_OK || r->status == SDD_E_TRUNCATED) {
        for (int j = 0; j < n; ++j)
            for (int e = 0; e < E; ++e) {
                const size_t o = (size_t)j * E + e;
                double mm[2], ss[2];
                finish(&r->sums[o * 4], r->nvalid[j], mm, ss);
                if (mean) { mean[2 * o] = mm[0]; mean[2 * o + 1] = mm[1]; }
                if (se) { se[2 * o] = ss[0]; se[2 * o + 1] = ss[1]; }
            }
        if (n_used)
            for (int j = 0; j < n; ++j) n_used[j] = r->n_used[j];
    }
    if (stats) {
        stats->queue_us = r->started ? us_since(r->t_submit, r->t_first) : 0.0;
        stats->latency_us = us_since(r->t_submit, r->t_done);
        stats->walks = r->walks;
        stats->truncated = r->truncated;
        stats->launches = r->launches;
        stats->status = r->status;
    }
    const sdd_status result = r->status;
    srv->free_slots.push_back(r->slot);
    srv->bytes_in_use -= r->bytes;
    srv->reqs.erase(it);
    delete r;
    return result;
}

extern "C" sdd_status sdd_server_cancel(sdd_server *srv, uint64_t id) {
    if (!srv) return fail(SDD_E_ARG, "srv is NULL");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(id);
    if (it == srv->reqs.end()) return fail(SDD_E_ARG, "unknown request id");
    SrvRequest *r = it->second;
    if (r->phase == 4) return SDD_OK;
    r->cancelled = true;
    // drop its queued pieces; pieces already on the GPU end it when they finish
    const size_t before = srv->runnable.size();
    srv->runnable.erase(std::remove_if(srv->runnable.begin(), srv->runnable.end(),
                                       [r](const SrvPiece &p) { return p.r == r; }),
                        srv->runnable.end());
    r->pieces_left -= (int)(before - srv->runnable.size());
    if (r->pieces_left == 0) {
        srv_finish(srv, r);
        srv->done_cv.notify_all();
    }
    return SDD_OK;
}

extern "C" sdd_status sdd_server_get_stats(sdd_server *srv, sdd_server_stats *out) {
    if (!srv || !out) return fail(SDD_E_ARG, "srv and out must not be NULL");
    std::lock_guard<std::mutex> lk(srv->mu);
    *out = srv->st;
    out->in_flight = (int32_t)srv->reqs.size();
    out->bytes_in_use = srv->bytes_in_use;
    return SDD_OK;
}

// ---------------------------------------------------------------------------
// Autotuning of the launch shape (sdd_autotune).

extern "C" sdd_status sdd_autotune(sdd_ctx *ctx, const double *nodes_xz, int32_t n_nodes,
                                   const int64_t *n_paths, double dt, uint64_t seed,
                                   const sdd_config *base, sdd_config *best,
                                   double *best_steps_per_s) {
    sdd_status st = check_call(ctx, n_nodes, n_paths, dt, base);
    if (st != SDD_OK) return st;
    if (n_nodes < 1 || !nodes_xz) return fail(SDD_E_ARG, "autotuning needs nodes");
    if (base && (base->block_threads || base->chunk_paths || base->guided_factor))
        return fail(SDD_E_ARG, "base must leave block_threads, chunk_paths and guided_factor automatic");
    sdd_config c;
    std::memset(&c, 0, sizeof(c));
    if (base) c = *base;
    const int blocks[] = {128, 192, 256};
    const int ks[] = {1, 2, 4, 8};  // guided factors
    std::vector<double> mean((size_t)n_nodes * ctx->E * 2), se(mean.size());
    double best_rate = -1.0;
    int best_b = 256, best_k = 2;
    const int saved_b = ctx->tune_block, saved_k = ctx->tune_k;
    const bool saved_read = ctx->tune_file_read;
    ctx->tune_file_read = true;  // time the candidates, not the cached choice
    for (int b : blocks)
        for (int k : ks) {
            ctx->tune_block = b;
            ctx->tune_k = k;
            double t = 1e30;
            uint64_t steps = 0;
            for (int rep = 0; rep < 2; ++rep) {
                sdd_stats sst;
                st = sdd_interface_values(ctx, nodes_xz, nullptr, n_nodes, n_paths, dt, seed, &c,
                                          mean.data(), se.data(), &sst);
                if (st != SDD_OK && st != SDD_E_TRUNCATED) {
                    ctx->tune_block = saved_b;
                    ctx->tune_k = saved_k;
                    ctx->tune_file_read = saved_read;
                    return st;
                }
                t = std::min(t, sst.kernel_ms);
                steps = sst.steps;
            }
            const double rate = (double)steps / (t * 1e-3);
            if (rate > best_rate) {
                best_rate = rate;
                best_b = b;
                best_k = k;
            }
        }
    ctx->tune_block = best_b;
    ctx->tune_k = best_k;
    if (const char *path = std::getenv("SDD_TUNE_CACHE")) {
        if (*path) {
            const bool f64 = c.precision == SDD_FP64;
            const std::string key = tune_key(ctx, kmax_for(ctx->K), ctx->M.gcode, f64, dt);
            if (FILE *f = std::fopen(path, "a")) {
                std::fprintf(f, "%s|%d %d\n", key.c_str(), best_b, best_k);
                std::fclose(f);
            }
        }
    }
    if (best) {
        *best = c;
        best->block_threads = best_b;
        best->chunk_paths = 0;
        best->guided_factor = best_k;
    }
    if (best_steps_per_s) *best_steps_per_s = best_rate;
    return SDD_OK;
}
