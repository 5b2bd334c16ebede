// Secondary fields, apparent resistivities and phases at measurement sites
// (Sec. 2.1: H^x = -(1/(i omega mu)) dE^y/dz, E^x = (1/sigma) dH^y/dz,
// rho = |E/H|^2 / (omega mu), phi = arg(E/H); Sec. 4.2: the solution at
// three points near the surface of each site, the z-derivative by the
// centred difference).
//
// Dimensionless form (lengths in units of L, kappa = omega mu sigma L^2,
// kappa_ref = omega mu sigma_ref L^2 for a reference conductivity): with u
// the primary field (E^y in TE, H^y in TM), u_z = (u(z0 + h) - u(z0 - h)) / 2h,
//   TE  rho / rho_ref = kappa_ref |u / u_z|^2,        phi = arg(-i u / u_z)
//   TM  rho / rho_ref = D^2 |u_z / u|^2 / kappa_ref,  phi = arg(u_z / u)
// where D = sigma_ref / sigma is the diffusion of the site's strip.  The
// three points' estimates and their real and imaginary parts are taken as
// independent, so the standard errors are first order (delta method) in the
// six real inputs.
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "sdd.h"
#include "sdd_internal.cuh"

namespace sdd {
namespace {

struct C2 {
    double re, im;
};
__device__ __forceinline__ C2 cmul(C2 a, C2 b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ C2 cdiv(C2 a, C2 b) {
    const double d = b.re * b.re + b.im * b.im;
    return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}

// Thread (site i, evaluation e).  mean, se: [3 n][E][2], the points of site
// i at rows 3 i (z0 - h), 3 i + 1 (z0), 3 i + 2 (z0 + h).  dsite: [n]
// diffusion of each site's strip (TM), nullptr for TE.
__global__ void mt_kernel(const double *mean, const double *se, int n, int E, double h,
                          const double *kref, const double *dsite, double *rho, double *phase,
                          double *rho_se, double *phase_se, double *u0_out, double *uz_out) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * E) return;
    const int i = idx / E, e = idx % E;
    const size_t r0 = ((size_t)(3 * i) * E + e) * 2, stride = (size_t)E * 2;
    const C2 um = {mean[r0], mean[r0 + 1]};
    const C2 a = {mean[r0 + stride], mean[r0 + stride + 1]};
    const C2 up = {mean[r0 + 2 * stride], mean[r0 + 2 * stride + 1]};
    const C2 uz = {(up.re - um.re) / (2.0 * h), (up.im - um.im) / (2.0 * h)};
    const bool te = dsite == nullptr;
    const C2 w = te ? cdiv(a, uz) : cdiv(uz, a);
    const double C = te ? kref[e] : dsite[i] * dsite[i] / kref[e];
    rho[idx] = C * (w.re * w.re + w.im * w.im);
    // TE: arg(-i w) = atan2(-Re w, Im w); TM: arg(w)
    phase[idx] = te ? atan2(-w.re, w.im) : atan2(w.im, w.re);
    if (u0_out) {
        u0_out[2 * idx] = a.re;
        u0_out[2 * idx + 1] = a.im;
    }
    if (uz_out) {
        uz_out[2 * idx] = uz.re;
        uz_out[2 * idx + 1] = uz.im;
    }
    if (rho_se || phase_se) {
        double vr = 0.0, vp = 0.0;
        for (int pt = 0; pt < 3; ++pt) {
            for (int comp = 0; comp < 2; ++comp) {
                const double s = se[r0 + pt * stride + comp];
                const C2 unit = comp == 0 ? C2{1.0, 0.0} : C2{0.0, 1.0};
                C2 dw;
                if (pt == 1) {
                    // a change of the centre value
                    dw = te ? cdiv(unit, uz) : cdiv(cmul(C2{-w.re, -w.im}, unit), a);
                } else {
                    // a change of u_z by +-unit / 2h
                    const double sg = (pt == 2 ? 1.0 : -1.0) / (2.0 * h);
                    const C2 de = {sg * unit.re, sg * unit.im};
                    dw = te ? cdiv(cmul(C2{-w.re, -w.im}, de), uz) : cdiv(de, a);
                }
                // d rho = 2 C Re(conj(w) dw), d phi = Im(dw / w)
                const double gr = 2.0 * C * (w.re * dw.re + w.im * dw.im);
                const double gp = cdiv(dw, w).im;
                vr += (gr * s) * (gr * s);
                vp += (gp * s) * (gp * s);
            }
        }
        if (rho_se) rho_se[idx] = sqrt(vr);
        if (phase_se) phase_se[idx] = sqrt(vp);
    }
}

sdd_status mt_cuda_error(cudaError_t e, const char *what) {
    return (sdd_status)report_error(SDD_E_CUDA, (std::string(what) + ": " + cudaGetErrorString(e)).c_str());
}

sdd_status mt_arg_error(const char *msg) { return (sdd_status)report_error(SDD_E_ARG, msg); }

#define MT_CUDA(call)                                                \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return mt_cuda_error(e_, #call);      \
    } while (0)

struct MtScratch {
    std::vector<void *> ptrs;
    cudaStream_t st = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    ~MtScratch() {
        for (void *p : ptrs) cudaFree(p);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        if (st) cudaStreamDestroy(st);
    }
    cudaError_t alloc(double **p, size_t count) {
        cudaError_t e = cudaMalloc((void **)p, (count ? count : 1) * sizeof(double));
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
};

// The kernel on host three-point estimates mean, se [3 n][E][2]; dsite
// [n] (TM) or nullptr (TE).  Adds its time, launch and copies to stats.
sdd_status mt_post(const double *mean, const double *se, int n_sites, int E, double h, const double *kappa_ref,
                   const double *dsite, double *rho, double *phase, double *rho_se, double *phase_se, double *u0,
                   double *uz, sdd_stats *stats) {
    MtScratch S;
    const bool tm = dsite != nullptr;
    double *dm, *ds, *dk, *dd = nullptr, *orho, *oph, *orse = nullptr, *opse = nullptr, *ou0 = nullptr,
                                                                                       *ouz = nullptr;
    const size_t nv = (size_t)3 * n_sites * E * 2, no = (size_t)n_sites * E;
    MT_CUDA(S.alloc(&dm, nv));
    MT_CUDA(S.alloc(&ds, nv));
    MT_CUDA(S.alloc(&dk, E));
    if (tm) MT_CUDA(S.alloc(&dd, n_sites));
    MT_CUDA(S.alloc(&orho, no));
    MT_CUDA(S.alloc(&oph, no));
    if (rho_se) MT_CUDA(S.alloc(&orse, no));
    if (phase_se) MT_CUDA(S.alloc(&opse, no));
    if (u0) MT_CUDA(S.alloc(&ou0, 2 * no));
    if (uz) MT_CUDA(S.alloc(&ouz, 2 * no));
    MT_CUDA(cudaStreamCreateWithFlags(&S.st, cudaStreamNonBlocking));
    MT_CUDA(cudaEventCreate(&S.ev[0]));
    MT_CUDA(cudaEventCreate(&S.ev[1]));
    cudaStream_t st = S.st;
    MT_CUDA(cudaMemcpyAsync(dm, mean, nv * sizeof(double), cudaMemcpyHostToDevice, st));
    MT_CUDA(cudaMemcpyAsync(ds, se, nv * sizeof(double), cudaMemcpyHostToDevice, st));
    MT_CUDA(cudaMemcpyAsync(dk, kappa_ref, E * sizeof(double), cudaMemcpyHostToDevice, st));
    if (tm) MT_CUDA(cudaMemcpyAsync(dd, dsite, n_sites * sizeof(double), cudaMemcpyHostToDevice, st));
    MT_CUDA(cudaEventRecord(S.ev[0], st));
    mt_kernel<<<(unsigned)((no + 127) / 128), 128, 0, st>>>(dm, ds, n_sites, E, h, dk, dd, orho, oph, orse,
                                                           opse, ou0, ouz);
    MT_CUDA(cudaGetLastError());
    MT_CUDA(cudaEventRecord(S.ev[1], st));
    MT_CUDA(cudaMemcpyAsync(rho, orho, no * sizeof(double), cudaMemcpyDeviceToHost, st));
    MT_CUDA(cudaMemcpyAsync(phase, oph, no * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (rho_se) MT_CUDA(cudaMemcpyAsync(rho_se, orse, no * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (phase_se) MT_CUDA(cudaMemcpyAsync(phase_se, opse, no * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (u0) MT_CUDA(cudaMemcpyAsync(u0, ou0, 2 * no * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (uz) MT_CUDA(cudaMemcpyAsync(uz, ouz, 2 * no * sizeof(double), cudaMemcpyDeviceToHost, st));
    MT_CUDA(cudaStreamSynchronize(st));
    if (stats) {
        float ms = 0.f;
        MT_CUDA(cudaEventElapsedTime(&ms, S.ev[0], S.ev[1]));
        stats->post_ms = ms;
        stats->launches += 1;
        stats->h2d_bytes += 2 * nv * sizeof(double) + E * sizeof(double) + (tm ? n_sites * sizeof(double) : 0);
        stats->d2h_bytes += no * sizeof(double) * (2 + (rho_se ? 1 : 0) + (phase_se ? 1 : 0) +
                                                   (u0 ? 2 : 0) + (uz ? 2 : 0));
    }
    return SDD_OK;
}

}  // namespace
}  // namespace sdd

using namespace sdd;

extern "C" sdd_status sdd_apparent_resistivity(sdd_ctx *ctx, const double *sites_xz, int32_t n_sites,
                                               double h, int64_t n_paths, const double *kappa_ref,
                                               double dt, uint64_t seed, const sdd_config *cfg,
                                               double *rho, double *phase, double *rho_se,
                                               double *phase_se, double *u0, double *uz,
                                               sdd_stats *stats) {
    if (!ctx) return mt_arg_error("ctx must not be NULL");
    if (n_sites < 0 || n_sites > SDD_MT_MAX_SITES) return mt_arg_error("n_sites must be in 0 .. SDD_MT_MAX_SITES");
    if (!(h > 0.0) || !std::isfinite(h)) return mt_arg_error("h must be finite and > 0");
    if (n_paths < 1 || n_paths > INT32_MAX) return mt_arg_error("n_paths must be in 1 .. 2^31-1");
    const int E = sdd_n_eval(ctx);
    if (!kappa_ref) return mt_arg_error("kappa_ref must not be NULL");
    for (int e = 0; e < E; ++e)
        if (!(kappa_ref[e] > 0.0) || !std::isfinite(kappa_ref[e]))
            return mt_arg_error("kappa_ref must be finite and > 0");
    if (stats) *stats = sdd_stats{};
    if (n_sites == 0) return SDD_OK;
    if (!sites_xz || !rho || !phase) return mt_arg_error("sites_xz, rho and phase must not be NULL");

    // the three points of each site under node ids 3 i, 3 i + 1, 3 i + 2
    const int np = 3 * n_sites;
    std::vector<double> pts(2 * (size_t)np), mean((size_t)np * E * 2), se((size_t)np * E * 2);
    std::vector<uint32_t> ids(np);
    std::vector<int64_t> paths(np, n_paths);
    std::vector<double> dsite(n_sites, 1.0);
    bool tm = false;
    for (int i = 0; i < n_sites; ++i) {
        for (int j = 0; j < 3; ++j) {
            pts[2 * (3 * i + j)] = sites_xz[2 * i];
            pts[2 * (3 * i + j) + 1] = sites_xz[2 * i + 1] + (j - 1) * h;
            ids[3 * i + j] = (uint32_t)(3 * i + j);
        }
        tm = ctx_site_diffusion(ctx, sites_xz[2 * i], &dsite[i]) != 0;
    }
    const sdd_status mc = sdd_interface_values(ctx, pts.data(), ids.data(), np, paths.data(), dt, seed,
                                               cfg, mean.data(), se.data(), stats);
    if (mc != SDD_OK && mc != SDD_E_TRUNCATED) return mc;

    const sdd_status r = mt_post(mean.data(), se.data(), n_sites, E, h, kappa_ref, tm ? dsite.data() : nullptr,
                                 rho, phase, rho_se, phase_se, u0, uz, stats);
    if (r != SDD_OK) return r;
    return mc;
}

extern "C" sdd_status sdd_apparent_from_values(const double *values, const double *se, int32_t n_sites,
                                               int32_t n_eval, double h, const double *kappa_ref,
                                               const double *d_site, double *rho, double *phase,
                                               double *rho_se, double *phase_se, double *u0, double *uz) {
    if (n_sites < 0 || n_sites > SDD_MT_MAX_SITES) return mt_arg_error("n_sites must be in 0 .. SDD_MT_MAX_SITES");
    if (n_eval < 1 || n_eval > SDD_MAX_EVAL) return mt_arg_error("n_eval must be in 1 .. SDD_MAX_EVAL");
    if (!(h > 0.0) || !std::isfinite(h)) return mt_arg_error("h must be finite and > 0");
    if (!kappa_ref) return mt_arg_error("kappa_ref must not be NULL");
    for (int e = 0; e < n_eval; ++e)
        if (!(kappa_ref[e] > 0.0) || !std::isfinite(kappa_ref[e]))
            return mt_arg_error("kappa_ref must be finite and > 0");
    if (n_sites == 0) return SDD_OK;
    if (!values || !se || !rho || !phase) return mt_arg_error("values, se, rho and phase must not be NULL");
    if (d_site)
        for (int i = 0; i < n_sites; ++i)
            if (!(d_site[i] > 0.0) || !std::isfinite(d_site[i])) return mt_arg_error("d_site must be finite and > 0");
    return mt_post(values, se, n_sites, n_eval, h, kappa_ref, d_site, rho, phase, rho_se, phase_se, u0, uz,
                   nullptr);
}
