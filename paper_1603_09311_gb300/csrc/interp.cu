// Interface values between Monte Carlo nodes (Sec. 5 of arXiv:1603.09311:
// the stochastic solution is computed at some points along an interface and
// the remaining interface values are interpolated).
//
// The paper gives no scheme; the one built here interpolates each real
// component of each evaluation in the arc length s along the interface
// polyline, piecewise linearly or by the natural cubic spline.  Both are
// linear in the knot values, v(s) = sum_j c_j(s) v_j, and the knots'
// estimates are independent, so the standard error carried to s is
// sqrt(sum_j c_j(s)^2 se_j^2).
//
// Kernels (all FP64; the work is small next to the walks that produce the
// knot values):
//   arc_kernel            arc length of the polyline, one CTA (chunk sums, a
//                         shared-memory scan, chunk prefixes)
//   spline_factor_kernel  Thomas forward coefficients of the natural-spline
//                         equations (one thread; at most 4096 knots)
//   spline_cols_kernel    G = the spline's second derivatives of every unit
//                         knot vector, one column per thread
//   interp_kernel         values and standard errors, one thread per target
//                         and component
//   scatter_kernel        the knots keep their own estimates
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "sdd.h"
#include "sdd_internal.cuh"

namespace sdd {
namespace {

constexpr int kArcThreads = 1024;

__global__ void __launch_bounds__(kArcThreads) arc_kernel(const double *p, int n, double *s) {
    __shared__ double part[kArcThreads];
    const int t = threadIdx.x;
    const int segs = n - 1;
    const int per = (segs + kArcThreads - 1) / kArcThreads;
    const int a = min(t * per, segs), b = min(a + per, segs);
    double acc = 0.0;
    for (int k = a; k < b; ++k) acc += hypot(p[2 * k + 2] - p[2 * k], p[2 * k + 3] - p[2 * k + 1]);
    part[t] = acc;
    __syncthreads();
    for (int off = 1; off < kArcThreads; off <<= 1) {
        const double v = t >= off ? part[t - off] : 0.0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    double run = t > 0 ? part[t - 1] : 0.0;
    if (t == 0) s[0] = 0.0;
    for (int k = a; k < b; ++k) {
        run += hypot(p[2 * k + 2] - p[2 * k], p[2 * k + 3] - p[2 * k + 1]);
        s[k + 1] = run;
    }
}

// The natural spline's second derivatives M solve, for the inner knots
// i = 1 .. n-2 (row r = i - 1), with h_i = s_{i+1} - s_i,
//   h_{i-1} M_{i-1} + 2 (h_{i-1} + h_i) M_i + h_i M_{i+1}
//       = 6 ((v_{i+1} - v_i) / h_i - (v_i - v_{i-1}) / h_{i-1}),
// M_0 = M_{n-1} = 0.  Thomas forward sweep: den_r = 2 (h_{i-1} + h_i) -
// h_{i-1} cp_{r-1}, cp_r = h_i / den_r.
__global__ void spline_factor_kernel(const double *s, int n, double *cp, double *den) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double prev = 0.0;
    for (int r = 0; r < n - 2; ++r) {
        const int i = r + 1;
        const double hl = s[i] - s[i - 1], hr = s[i + 1] - s[i];
        const double d = 2.0 * (hl + hr) - (r > 0 ? hl * prev : 0.0);
        den[r] = d;
        prev = hr / d;
        cp[r] = prev;
    }
}

// Knot spacings must be positive (arc lengths of distinct nodes can still
// round to equal sums): *err = 1 otherwise.
__global__ void knots_check_kernel(const double *s, int n, int *err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
    if (i < n && !(s[i] > s[i - 1])) atomicExch(err, 1);
}

// Column j of G [n][n]: M(e_j), the second derivatives of the natural spline
// through the unit vector e_j.  The right-hand side of row r (knot i = r + 1)
// is non-zero for i in {j - 1, j, j + 1} only.
__global__ void spline_cols_kernel(const double *s, int n, const double *cp, const double *den,
                                   double *G) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int m = n - 2;
    G[j] = 0.0;
    G[(size_t)(n - 1) * n + j] = 0.0;
    double dprev = 0.0;
    for (int r = 0; r < m; ++r) {
        const int i = r + 1;
        const double hl = s[i] - s[i - 1], hr = s[i + 1] - s[i];
        double rhs = 0.0;
        if (j == i - 1) rhs = 6.0 / hl;
        else if (j == i) rhs = -(6.0 / hl + 6.0 / hr);
        else if (j == i + 1) rhs = 6.0 / hr;
        const double d = (rhs - (r > 0 ? hl * dprev : 0.0)) / den[r];
        G[(size_t)i * n + j] = d;
        dprev = d;
    }
    double xnext = 0.0;
    for (int r = m - 1; r >= 0; --r) {
        const size_t o = (size_t)(r + 1) * n + j;
        const double x = G[o] - (r < m - 1 ? cp[r] * xnext : 0.0);
        G[o] = x;
        xnext = x;
    }
}

// Thread (target q, component c).  The target's segment is the largest
// i <= nk - 2 with s_i <= t; with a = (s_{i+1} - t) / h and b = (t - s_i) / h
//   linear  c_i = a, c_{i+1} = b
//   spline  c_j = a [j = i] + b [j = i + 1]
//                 + (a^3 - a) h^2 / 6 G[i][j] + (b^3 - b) h^2 / 6 G[i+1][j]
// (G == nullptr selects the linear interpolant).
__global__ void interp_kernel(const double *sk, int nk, const double *G, const double *v,
                              const double *se, int V, const double *t, int nt, double *ov,
                              double *ose) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)nt * V) return;
    const int q = (int)(idx / V), c = (int)(idx % V);
    const double x = t[q];
    int lo = 0, hi = nk - 2;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sk[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    const int i = lo;
    const double h = sk[i + 1] - sk[i];
    const double a = (sk[i + 1] - x) / h, b = (x - sk[i]) / h;
    double val, var = 0.0;
    if (!G) {
        const double v0 = v[(size_t)i * V + c], v1 = v[(size_t)(i + 1) * V + c];
        val = a * v0 + b * v1;
        if (se) {
            const double e0 = a * se[(size_t)i * V + c], e1 = b * se[(size_t)(i + 1) * V + c];
            var = e0 * e0 + e1 * e1;
        }
    } else {
        const double al = (a * a * a - a) * h * h / 6.0, be = (b * b * b - b) * h * h / 6.0;
        const double *gi = G + (size_t)i * nk, *gi1 = G + (size_t)(i + 1) * nk;
        val = 0.0;
        for (int j = 0; j < nk; ++j) {
            double cj = al * gi[j] + be * gi1[j];
            if (j == i) cj += a;
            if (j == i + 1) cj += b;
            val += cj * v[(size_t)j * V + c];
            if (se) {
                const double e = cj * se[(size_t)j * V + c];
                var += e * e;
            }
        }
    }
    ov[idx] = val;
    if (ose) ose[idx] = sqrt(var);
}

__global__ void gather_kernel(const double *s, const int32_t *idx, int nk, double *out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < nk) out[j] = s[idx[j]];
}

__global__ void scatter_kernel(const double *kv, const double *kse, const int32_t *idx, int nk,
                               int V, double *ov, double *ose) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)nk * V) return;
    const int j = (int)(e / V), c = (int)(e % V);
    ov[(size_t)idx[j] * V + c] = kv[e];
    ose[(size_t)idx[j] * V + c] = kse[e];
}

// Device allocations of one call, freed on every return path.
struct Scratch {
    std::vector<void *> ptrs;
    ~Scratch() {
        for (void *p : ptrs) cudaFree(p);
    }
    template <class T>
    cudaError_t alloc(T **p, size_t count) {
        *p = nullptr;
        if (count == 0) count = 1;
        cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
};

#define INTERP_CUDA(call)                                            \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return cuda_error(e_, #call);         \
    } while (0)

sdd_status cuda_error(cudaError_t e, const char *what) {
    return (sdd_status)report_error(SDD_E_CUDA, (std::string(what) + ": " + cudaGetErrorString(e)).c_str());
}

sdd_status arg_error(const char *msg) { return (sdd_status)report_error(SDD_E_ARG, msg); }

// Interpolation of device knot data to device targets on stream st.  The
// knot check's flag is copied to *h_err, valid once st has been
// synchronised.
sdd_status run_interp(const double *d_sk, int nk, const double *d_v, const double *d_se, int V,
                      const double *d_t, int nt, int kind, double *d_ov, double *d_ose,
                      Scratch &S, cudaStream_t st, int *h_err) {
    int *err;
    INTERP_CUDA(S.alloc(&err, 1));
    INTERP_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    knots_check_kernel<<<(nk + 127) / 128, 128, 0, st>>>(d_sk, nk, err);
    INTERP_CUDA(cudaGetLastError());
    const double *G = nullptr;
    if (kind == SDD_INTERP_SPLINE && nk > 2) {
        double *g, *cp, *den;
        INTERP_CUDA(S.alloc(&g, (size_t)nk * nk));
        INTERP_CUDA(S.alloc(&cp, (size_t)nk));
        INTERP_CUDA(S.alloc(&den, (size_t)nk));
        spline_factor_kernel<<<1, 32, 0, st>>>(d_sk, nk, cp, den);
        INTERP_CUDA(cudaGetLastError());
        spline_cols_kernel<<<(nk + 127) / 128, 128, 0, st>>>(d_sk, nk, cp, den, g);
        INTERP_CUDA(cudaGetLastError());
        G = g;
    }
    const long long total = (long long)nt * V;
    if (total > 0) {
        const int threads = 128;
        interp_kernel<<<(unsigned)((total + threads - 1) / threads), threads, 0, st>>>(
            d_sk, nk, G, d_v, d_se, V, d_t, nt, d_ov, d_ose);
        INTERP_CUDA(cudaGetLastError());
    }
    INTERP_CUDA(cudaMemcpyAsync(h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    return SDD_OK;
}

}  // namespace
}  // namespace sdd

using namespace sdd;

extern "C" sdd_status sdd_interpolate(const double *knots_s, int32_t n_knots, const double *values,
                                      const double *se, int32_t n_vals, const double *targets_s,
                                      int32_t n_targets, int32_t kind, double *out_values,
                                      double *out_se) {
    if (kind != SDD_INTERP_LINEAR && kind != SDD_INTERP_SPLINE)
        return arg_error("kind must be SDD_INTERP_LINEAR or SDD_INTERP_SPLINE");
    if (n_knots < 2) return arg_error("n_knots must be at least 2");
    if (kind == SDD_INTERP_SPLINE && n_knots > SDD_INTERP_MAX_SPLINE_KNOTS)
        return arg_error("n_knots exceeds SDD_INTERP_MAX_SPLINE_KNOTS for the spline");
    if (n_vals < 1) return arg_error("n_vals must be at least 1");
    if (n_targets < 0) return arg_error("n_targets must not be negative");
    if (!knots_s || !values || (n_targets > 0 && (!targets_s || !out_values)))
        return arg_error("knots_s, values, targets_s and out_values must not be NULL");
    for (int i = 0; i < n_knots; ++i) {
        if (!std::isfinite(knots_s[i])) return arg_error("knots must be finite");
        if (i > 0 && !(knots_s[i] > knots_s[i - 1])) return arg_error("knots must be strictly increasing");
    }
    for (int q = 0; q < n_targets; ++q)
        if (!(targets_s[q] >= knots_s[0] && targets_s[q] <= knots_s[n_knots - 1]))
            return arg_error("targets must lie within [knots_s[0], knots_s[n_knots - 1]]");
    if (n_targets == 0) return SDD_OK;
    const bool with_se = se != nullptr && out_se != nullptr;
    const size_t kb = (size_t)n_knots * n_vals, tb = (size_t)n_targets * n_vals;
    Scratch S;
    double *sk, *v, *e = nullptr, *t, *ov, *oe = nullptr;
    INTERP_CUDA(S.alloc(&sk, n_knots));
    INTERP_CUDA(S.alloc(&v, kb));
    INTERP_CUDA(S.alloc(&t, n_targets));
    INTERP_CUDA(S.alloc(&ov, tb));
    if (with_se) {
        INTERP_CUDA(S.alloc(&e, kb));
        INTERP_CUDA(S.alloc(&oe, tb));
    }
    cudaStream_t st;
    INTERP_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamDestroy(s); }
    } guard{st};
    INTERP_CUDA(cudaMemcpyAsync(sk, knots_s, n_knots * sizeof(double), cudaMemcpyHostToDevice, st));
    INTERP_CUDA(cudaMemcpyAsync(v, values, kb * sizeof(double), cudaMemcpyHostToDevice, st));
    INTERP_CUDA(cudaMemcpyAsync(t, targets_s, n_targets * sizeof(double), cudaMemcpyHostToDevice, st));
    if (with_se) INTERP_CUDA(cudaMemcpyAsync(e, se, kb * sizeof(double), cudaMemcpyHostToDevice, st));
    int h_err = 0;
    sdd_status r = run_interp(sk, n_knots, v, e, n_vals, t, n_targets, kind, ov, oe, S, st, &h_err);
    if (r != SDD_OK) return r;
    INTERP_CUDA(cudaMemcpyAsync(out_values, ov, tb * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (with_se) INTERP_CUDA(cudaMemcpyAsync(out_se, oe, tb * sizeof(double), cudaMemcpyDeviceToHost, st));
    INTERP_CUDA(cudaStreamSynchronize(st));
    if (h_err) return arg_error("knots must be strictly increasing");
    return SDD_OK;
}

extern "C" sdd_status sdd_interface_values_interp(sdd_ctx *ctx, const double *nodes_xz,
                                                  int32_t n_nodes, int32_t stride, int64_t n_paths,
                                                  int32_t kind, double dt, uint64_t seed,
                                                  const sdd_config *cfg, double *mean, double *se,
                                                  sdd_stats *stats) {
    if (!ctx) return arg_error("ctx must not be NULL");
    if (kind != SDD_INTERP_LINEAR && kind != SDD_INTERP_SPLINE)
        return arg_error("kind must be SDD_INTERP_LINEAR or SDD_INTERP_SPLINE");
    if (n_nodes < 2 || n_nodes > SDD_INTERP_MAX_NODES)
        return arg_error("n_nodes must be in 2 .. SDD_INTERP_MAX_NODES");
    if (stride < 1) return arg_error("stride must be at least 1");
    if (n_paths < 1 || n_paths > INT32_MAX) return arg_error("n_paths must be in 1 .. 2^31-1");
    if (!nodes_xz || !mean || !se) return arg_error("nodes_xz, mean and se must not be NULL");
    for (int i = 1; i < n_nodes; ++i)
        if (nodes_xz[2 * i] == nodes_xz[2 * i - 2] && nodes_xz[2 * i + 1] == nodes_xz[2 * i - 1])
            return arg_error("consecutive interface nodes must differ");
    std::vector<int32_t> kidx;
    for (int i = 0; i < n_nodes; i += stride) kidx.push_back(i);
    if (kidx.back() != n_nodes - 1) kidx.push_back(n_nodes - 1);
    const int nk = (int)kidx.size();
    if (kind == SDD_INTERP_SPLINE && nk > SDD_INTERP_MAX_SPLINE_KNOTS)
        return arg_error("too many Monte Carlo nodes for the spline (SDD_INTERP_MAX_SPLINE_KNOTS)");
    const int E = sdd_n_eval(ctx), V = 2 * E;

    // Monte Carlo at the knots, each under its index along the polyline as
    // RNG node id (the values sdd_interface_values gives those nodes in a
    // call on the whole polyline)
    std::vector<double> knodes(2 * (size_t)nk), kmean((size_t)nk * V), kse((size_t)nk * V);
    std::vector<uint32_t> kid(nk);
    std::vector<int64_t> kpaths(nk, n_paths);
    for (int j = 0; j < nk; ++j) {
        knodes[2 * j] = nodes_xz[2 * (size_t)kidx[j]];
        knodes[2 * j + 1] = nodes_xz[2 * (size_t)kidx[j] + 1];
        kid[j] = (uint32_t)kidx[j];
    }
    const sdd_status mc = sdd_interface_values(ctx, knodes.data(), kid.data(), nk, kpaths.data(), dt,
                                               seed, cfg, kmean.data(), kse.data(), stats);
    if (mc != SDD_OK && mc != SDD_E_TRUNCATED) return mc;

    Scratch S;
    double *p, *s, *sk, *kv, *ke, *ov, *oe;
    int32_t *di;
    const size_t ob = (size_t)n_nodes * V;
    INTERP_CUDA(S.alloc(&p, 2 * (size_t)n_nodes));
    INTERP_CUDA(S.alloc(&s, (size_t)n_nodes));
    INTERP_CUDA(S.alloc(&sk, (size_t)nk));
    INTERP_CUDA(S.alloc(&di, (size_t)nk));
    INTERP_CUDA(S.alloc(&kv, (size_t)nk * V));
    INTERP_CUDA(S.alloc(&ke, (size_t)nk * V));
    INTERP_CUDA(S.alloc(&ov, ob));
    INTERP_CUDA(S.alloc(&oe, ob));
    cudaStream_t st;
    INTERP_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamDestroy(s); }
    } guard{st};
    INTERP_CUDA(cudaMemcpyAsync(p, nodes_xz, 2 * (size_t)n_nodes * sizeof(double), cudaMemcpyHostToDevice, st));
    INTERP_CUDA(cudaMemcpyAsync(di, kidx.data(), nk * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    INTERP_CUDA(cudaMemcpyAsync(kv, kmean.data(), (size_t)nk * V * sizeof(double), cudaMemcpyHostToDevice, st));
    INTERP_CUDA(cudaMemcpyAsync(ke, kse.data(), (size_t)nk * V * sizeof(double), cudaMemcpyHostToDevice, st));
    cudaEvent_t ev[2];
    INTERP_CUDA(cudaEventCreate(&ev[0]));
    struct EventGuard {
        cudaEvent_t *e;
        int n = 0;
        ~EventGuard() {
            for (int i = 0; i < n; ++i) cudaEventDestroy(e[i]);
        }
    } eg{ev, 1};
    INTERP_CUDA(cudaEventCreate(&ev[1]));
    eg.n = 2;
    INTERP_CUDA(cudaEventRecord(ev[0], st));
    arc_kernel<<<1, kArcThreads, 0, st>>>(p, n_nodes, s);
    INTERP_CUDA(cudaGetLastError());
    gather_kernel<<<(nk + 127) / 128, 128, 0, st>>>(s, di, nk, sk);
    INTERP_CUDA(cudaGetLastError());
    int h_err = 0;
    sdd_status r = run_interp(sk, nk, kv, ke, V, s, n_nodes, kind, ov, oe, S, st, &h_err);
    if (r != SDD_OK) return r;
    const long long kt = (long long)nk * V;
    scatter_kernel<<<(unsigned)((kt + 127) / 128), 128, 0, st>>>(kv, ke, di, nk, V, ov, oe);
    INTERP_CUDA(cudaGetLastError());
    INTERP_CUDA(cudaEventRecord(ev[1], st));
    INTERP_CUDA(cudaMemcpyAsync(mean, ov, ob * sizeof(double), cudaMemcpyDeviceToHost, st));
    INTERP_CUDA(cudaMemcpyAsync(se, oe, ob * sizeof(double), cudaMemcpyDeviceToHost, st));
    INTERP_CUDA(cudaStreamSynchronize(st));
    if (h_err) return arg_error("the arc lengths of the Monte Carlo nodes must be strictly increasing");
    if (stats) {
        float ms = 0.f;
        INTERP_CUDA(cudaEventElapsedTime(&ms, ev[0], ev[1]));
        stats->post_ms = ms;
        // arc length, knot gather, knot check, [spline factor, spline columns], interpolation, scatter
        stats->launches += (kind == SDD_INTERP_SPLINE && nk > 2) ? 7 : 5;
        stats->h2d_bytes += 2 * (uint64_t)n_nodes * sizeof(double) + (uint64_t)nk * sizeof(int32_t) +
                            2 * (uint64_t)nk * V * sizeof(double);
        stats->d2h_bytes += 2 * (uint64_t)ob * sizeof(double) + sizeof(int);
    }
    return mc;
}
