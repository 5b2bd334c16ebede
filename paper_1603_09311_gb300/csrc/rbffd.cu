// RBF-FD sub-domain solver (Sec. 3.2 of arXiv:1603.09311): once the
// interface values are known, a sub-domain is solved on its own nodes with
// radial-basis-function finite differences.
//
// At node x_0 with stencil x_1 .. x_n (the node and its n - 1 nearest
// neighbours), the weights of an operator L solve A w = b with
// A_ij = phi(|x_i - x_j|) and b_j = L phi(|x - x_j|) at x_0, for the
// multiquadric phi(r) = sqrt(1 + (eps r)^2).  The operator is the Laplacian
// (the sum of the paper's d^2/dx^2 and d^2/dz^2 matrices; the weights are
// linear in b): Lap phi = (2 eps^2 + eps^4 r^2) / phi^3 in two dimensions.
// Every unknown node i gets the equation
//     sum_{j in stencil(i)} w_ij u_j - i kappa_i u_i = 0,
// the Dirichlet nodes' terms moved to the right-hand side, and the sparse
// complex system is solved by BiCGStab with a Jacobi preconditioner.
//
// Kernels (FP64, this unit compiled without FMA contraction so that the
// squared distances of the neighbour search round as in plain arithmetic):
//   cell_*, knn_kernel  each node's nearest nodes by (squared distance,
//                    index): nodes binned into a cell grid, one thread per
//                    node scanning rings of cells
//   weights_kernel   one thread per node: the n x n multiquadric system,
//                    Gaussian elimination with partial pivoting
//   assemble_kernel  one thread per unknown: the row (ELL, n slots, column
//                    -1 for a Dirichlet neighbour), the diagonal and the
//                    right-hand side
//   BiCGStab         five launches per iteration: element-wise updates and
//                    ELL matrix-vector products, each dot product finished
//                    by the last block of its launch (block partials summed
//                    in block order), scalars on the device; batches of 8
//                    iterations replayed as a CUDA graph, the host reading
//                    the stop flag after each batch
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "sdd.h"
#include "sdd_internal.cuh"

namespace sdd {
namespace {

constexpr int kMaxStencil = 16;
constexpr int kDotThreads = 256;
constexpr int kDotBlocks = 1024;

struct Z {
    double re, im;
};
__device__ __forceinline__ Z zadd(Z a, Z b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ Z zsub(Z a, Z b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ Z zmul(Z a, Z b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ Z zdiv(Z a, Z b) {
    const double d = b.re * b.re + b.im * b.im;
    return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
// conj(a) b
__device__ __forceinline__ Z zcdot(Z a, Z b) { return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re}; }

__device__ __forceinline__ double mq(double r2, double eps) { return sqrt(1.0 + eps * eps * r2); }

// Nearest-neighbour search on a grid of square cells of side c over the
// nodes' bounding box: nodes are binned (count, scan, fill), then each node
// scans rings of cells around its own (ring R: Chebyshev cell distance R).
// Every node in ring R + 1 or beyond is at least R c away, so the search
// stops after ring R once the list is full and (R c)^2 exceeds its last
// squared distance (with a relative margin of 1e-9 for the binning's
// rounding).  The order is (squared distance, index), as a scan of all nodes
// gives.
struct CellGrid {
    double x0, z0, c;
    int gx, gz;
};

__device__ __forceinline__ int cell_x(const CellGrid &g, double x) {
    return min(max((int)floor((x - g.x0) / g.c), 0), g.gx - 1);
}
__device__ __forceinline__ int cell_z(const CellGrid &g, double z) {
    return min(max((int)floor((z - g.z0) / g.c), 0), g.gz - 1);
}

__global__ void cell_count_kernel(const double *p, int n, CellGrid g, int32_t *cell, int32_t *count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int id = cell_z(g, p[2 * i + 1]) * g.gx + cell_x(g, p[2 * i]);
    cell[i] = id;
    atomicAdd(&count[id], 1);
}

// start[0 .. m] = exclusive prefix sums of count[0 .. m-1] (one CTA).
__global__ void __launch_bounds__(1024) cell_scan_kernel(const int32_t *count, int m, int32_t *start) {
    __shared__ int32_t part[1024];
    const int t = threadIdx.x;
    const int per = (m + 1023) / 1024;
    const int a = min(t * per, m), b = min(a + per, m);
    int32_t acc = 0;
    for (int k = a; k < b; ++k) acc += count[k];
    part[t] = acc;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int32_t v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int32_t run = t > 0 ? part[t - 1] : 0;
    for (int k = a; k < b; ++k) {
        start[k] = run;
        run += count[k];
    }
    if (t == 1023) start[m] = part[1023];
}

__global__ void cell_fill_kernel(const int32_t *cell, int n, int32_t *cursor, int32_t *list) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    list[atomicAdd(&cursor[cell[i]], 1)] = i;
}

__device__ __forceinline__ bool before(double d2, int j, double bd, int bj) {
    return d2 < bd || (d2 == bd && j < bj);
}

__global__ void knn_kernel(const double *p, int n, int ns, CellGrid g, const int32_t *start,
                           const int32_t *list, int32_t *st) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double bd[kMaxStencil];
    int bi[kMaxStencil];
    int cnt = 0;
    const double xi = p[2 * i], zi = p[2 * i + 1];
    const int cx = cell_x(g, xi), cz = cell_z(g, zi);
    const int rmax = max(g.gx, g.gz);
    for (int R = 0; R <= rmax; ++R) {
        for (int dz = -R; dz <= R; ++dz) {
            const int iz = cz + dz;
            if (iz < 0 || iz >= g.gz) continue;
            const int step = (dz == -R || dz == R) ? 1 : 2 * R;
            for (int dx = -R; dx <= R; dx += (step > 0 ? step : 1)) {
                const int ix = cx + dx;
                if (ix < 0 || ix >= g.gx) continue;
                const int id = iz * g.gx + ix;
                for (int q = start[id]; q < start[id + 1]; ++q) {
                    const int j = list[q];
                    const double ddx = p[2 * j] - xi, ddz = p[2 * j + 1] - zi;
                    const double d2 = ddx * ddx + ddz * ddz;
                    if (cnt == ns && !before(d2, j, bd[ns - 1], bi[ns - 1])) continue;
                    int k = cnt < ns ? cnt++ : ns - 1;
                    while (k > 0 && before(d2, j, bd[k - 1], bi[k - 1])) {
                        bd[k] = bd[k - 1];
                        bi[k] = bi[k - 1];
                        --k;
                    }
                    bd[k] = d2;
                    bi[k] = j;
                }
            }
        }
        if (cnt == ns) {
            const double rc = R * g.c;
            if (rc * rc * (1.0 - 1e-9) > bd[ns - 1]) break;
        }
    }
    for (int k = 0; k < ns; ++k) st[(size_t)i * ns + k] = bi[k];
}

// Weights of node i, w[i][k] for stencil entry k.  *err = 1 on a zero pivot
// (coincident nodes).
__global__ void weights_kernel(const double *p, int n, const int32_t *st, int ns, double eps,
                               double *w, int *err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double A[kMaxStencil][kMaxStencil + 1];
    const double xi = p[2 * i], zi = p[2 * i + 1];
    for (int a = 0; a < ns; ++a) {
        const int ja = st[(size_t)i * ns + a];
        const double xa = p[2 * ja], za = p[2 * ja + 1];
        for (int b = 0; b < ns; ++b) {
            const int jb = st[(size_t)i * ns + b];
            const double r = hypot(xa - p[2 * jb], za - p[2 * jb + 1]);
            A[a][b] = mq(r * r, eps);
        }
        const double r = hypot(xa - xi, za - zi);
        const double ph = mq(r * r, eps);
        A[a][ns] = (2.0 * eps * eps + eps * eps * eps * eps * r * r) / (ph * ph * ph);
    }
    for (int c = 0; c < ns; ++c) {
        int piv = c;
        double best = fabs(A[c][c]);
        for (int r = c + 1; r < ns; ++r)
            if (fabs(A[r][c]) > best) {
                best = fabs(A[r][c]);
                piv = r;
            }
        if (!(best > 0.0)) {
            atomicExch(err, 1);
            return;
        }
        if (piv != c)
            for (int k = c; k <= ns; ++k) {
                const double t = A[c][k];
                A[c][k] = A[piv][k];
                A[piv][k] = t;
            }
        for (int r = c + 1; r < ns; ++r) {
            const double f = A[r][c] / A[c][c];
            for (int k = c; k <= ns; ++k) A[r][k] -= f * A[c][k];
        }
    }
    for (int c = ns - 1; c >= 0; --c) {
        double s = A[c][ns];
        for (int k = c + 1; k < ns; ++k) s -= A[c][k] * A[k][ns];
        A[c][ns] = s / A[c][c];
    }
    for (int k = 0; k < ns; ++k) w[(size_t)i * ns + k] = A[k][ns];
}

// Row r (node unk[r]): ELL slots k-major (ew[k nu + r], ecol[k nu + r]),
// the reciprocal of the diagonal d = w_ii - i kappa_i (the Jacobi
// preconditioner), right-hand side -sum_{Dirichlet j} w_ij u_j.
__global__ void assemble_kernel(const int32_t *unk, const int32_t *pos, int nu, const int32_t *st,
                                const double *w, int ns, const double *kappa, const double *vals,
                                double *ew, int32_t *ecol, Z *dinv, Z *rhs) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nu) return;
    const int i = unk[r];
    Z b = {0.0, 0.0};
    double wii = 0.0;
    for (int k = 0; k < ns; ++k) {
        const int j = st[(size_t)i * ns + k];
        const double wij = w[(size_t)i * ns + k];
        const int c = pos[j];
        ew[(size_t)k * nu + r] = wij;
        ecol[(size_t)k * nu + r] = c;
        if (c < 0) {
            b.re -= wij * vals[2 * j];
            b.im -= wij * vals[2 * j + 1];
        }
        if (j == i) wii = wij;
    }
    dinv[r] = zdiv(Z{1.0, 0.0}, Z{wii, -kappa[i]});
    rhs[r] = b;
}

// y = K x: sum over the slots, minus i kappa x on the diagonal
__global__ void spmv_kernel(const double *ew, const int32_t *ecol, int nu, int ns, const int32_t *unk,
                            const double *kappa, const Z *x, Z *y) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nu) return;
    Z acc = {0.0, 0.0};
    for (int k = 0; k < ns; ++k) {
        const int c = ecol[(size_t)k * nu + r];
        if (c >= 0) {
            const double wv = ew[(size_t)k * nu + r];
            acc.re += wv * x[c].re;
            acc.im += wv * x[c].im;
        }
    }
    const double kap = kappa[unk[r]];
    // - i kappa x = kappa (x.im, -x.re)
    acc.re += kap * x[r].im;
    acc.im -= kap * x[r].re;
    y[r] = acc;
}

// Block partials of sum conj(a_i) b_i (and of sum conj(a_i) c_i when c).
__global__ void __launch_bounds__(kDotThreads) dot_partial_kernel(const Z *a, const Z *b, const Z *c,
                                                                  int n, Z *part_b, Z *part_c) {
    __shared__ Z sb[kDotThreads], sc[kDotThreads];
    Z ab = {0.0, 0.0}, ac = {0.0, 0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        ab = zadd(ab, zcdot(a[i], b[i]));
        if (c) ac = zadd(ac, zcdot(a[i], c[i]));
    }
    sb[threadIdx.x] = ab;
    sc[threadIdx.x] = ac;
    __syncthreads();
    for (int off = kDotThreads / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) {
            sb[threadIdx.x] = zadd(sb[threadIdx.x], sb[threadIdx.x + off]);
            sc[threadIdx.x] = zadd(sc[threadIdx.x], sc[threadIdx.x + off]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part_b[blockIdx.x] = sb[0];
        if (c) part_c[blockIdx.x] = sc[0];
    }
}

// Device-side BiCGStab scalars.  stop: 0 running, 1 converged, 2 breakdown.
// ticket: the block counter of the launch that is finishing a dot product.
struct Scal {
    Z rho, alpha, omega, beta;
    double rnorm2, bnorm2, tol2;
    int iter, stop;
    unsigned ticket;
};

// Block reduction of one or two complex values; thread 0 writes the block's
// partials, then takes a ticket.  Returns true in every thread of the last
// block to finish, which then holds all partials (read past L1).
__device__ bool partial_and_ticket(Z v0, Z v1, bool two, Z *part0, Z *part1, unsigned *ticket) {
    __shared__ Z s0[kDotThreads], s1[kDotThreads];
    __shared__ bool last;
    s0[threadIdx.x] = v0;
    s1[threadIdx.x] = v1;
    __syncthreads();
    for (int off = kDotThreads / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) {
            s0[threadIdx.x] = zadd(s0[threadIdx.x], s0[threadIdx.x + off]);
            if (two) s1[threadIdx.x] = zadd(s1[threadIdx.x], s1[threadIdx.x + off]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part0[blockIdx.x] = s0[0];
        if (two) part1[blockIdx.x] = s1[0];
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    return last;
}

// The sum of the partials in block order (the last block only).
__device__ Z sum_partials(const Z *part, int np) {
    __shared__ Z s[kDotThreads];
    Z acc = {0.0, 0.0};
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
        const double2 v = __ldcg(reinterpret_cast<const double2 *>(part) + i);
        acc = zadd(acc, Z{v.x, v.y});
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int off = kDotThreads / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) s[threadIdx.x] = zadd(s[threadIdx.x], s[threadIdx.x + off]);
        __syncthreads();
    }
    const Z out = s[0];
    __syncthreads();
    return out;
}

__device__ __forceinline__ Z spmv_row(const double *ew, const int32_t *ecol, int nu, int ns, double kap,
                                      const Z *x, int r) {
    Z acc = {0.0, 0.0};
    for (int k = 0; k < ns; ++k) {
        const int c = ecol[(size_t)k * nu + r];
        if (c >= 0) {
            const double wv = ew[(size_t)k * nu + r];
            acc.re += wv * x[c].re;
            acc.im += wv * x[c].im;
        }
    }
    // - i kappa x = kappa (x.im, -x.re)
    acc.re += kap * x[r].im;
    acc.im -= kap * x[r].re;
    return acc;
}

// One BiCGStab iteration is five launches (grid-stride loops over the rows,
// the dot products finished by each launch's last block; dinv = 1 / d):
//   update_p      p = r + beta (p - omega v),  y = p / d
//   spmv_alpha    v = K y,  alpha = rho / <r^, v>
//   update_s      s = r - alpha v,  z = s / d
//   spmv_omega    t = K z,  omega = <t, s> / <t, t>  (t = 0: s = 0, omega = 0)
//   update_x      x += alpha y + omega z,  r = s - omega t,  |r|^2 and the
//                 stop test, rho' = <r^, r>,  beta = (rho' / rho)(alpha / omega)
// Every launch does nothing once stop is set.
__global__ void __launch_bounds__(kDotThreads) update_p_kernel(int n, const Scal *S, const Z *r, const Z *v,
                                                               const Z *dinv, Z *p, Z *y) {
    if (S->stop) return;
    const Z beta = S->beta, omega = S->omega;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const Z pi = zadd(r[i], zmul(beta, zsub(p[i], zmul(omega, v[i]))));
        p[i] = pi;
        y[i] = zmul(pi, dinv[i]);
    }
}

__global__ void __launch_bounds__(kDotThreads) spmv_alpha_kernel(const double *ew, const int32_t *ecol, int nu,
                                                                 int ns, const int32_t *unk, const double *kappa,
                                                                 const Z *y, const Z *rh, Z *v, Z *part,
                                                                 Scal *S) {
    if (S->stop) return;
    Z acc = {0.0, 0.0};
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nu; r += gridDim.x * blockDim.x) {
        const Z vr = spmv_row(ew, ecol, nu, ns, kappa[unk[r]], y, r);
        v[r] = vr;
        acc = zadd(acc, zcdot(rh[r], vr));
    }
    if (!partial_and_ticket(acc, Z{0.0, 0.0}, false, part, nullptr, &S->ticket)) return;
    const Z rv = sum_partials(part, gridDim.x);
    if (threadIdx.x == 0) {
        S->ticket = 0;
        if (rv.re == 0.0 && rv.im == 0.0) S->stop = 2;
        else S->alpha = zdiv(S->rho, rv);
    }
}

__global__ void __launch_bounds__(kDotThreads) update_s_kernel(int n, const Scal *S, const Z *r, const Z *v,
                                                               const Z *dinv, Z *s, Z *z) {
    if (S->stop) return;
    const Z alpha = S->alpha;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const Z si = zsub(r[i], zmul(alpha, v[i]));
        s[i] = si;
        z[i] = zmul(si, dinv[i]);
    }
}

__global__ void __launch_bounds__(kDotThreads) spmv_omega_kernel(const double *ew, const int32_t *ecol, int nu,
                                                                 int ns, const int32_t *unk, const double *kappa,
                                                                 const Z *z, const Z *s, Z *t, Z *part0,
                                                                 Z *part1, Scal *S) {
    if (S->stop) return;
    Z ts = {0.0, 0.0}, tt = {0.0, 0.0};
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nu; r += gridDim.x * blockDim.x) {
        const Z tr = spmv_row(ew, ecol, nu, ns, kappa[unk[r]], z, r);
        t[r] = tr;
        ts = zadd(ts, zcdot(tr, s[r]));
        tt = zadd(tt, zcdot(tr, tr));
    }
    if (!partial_and_ticket(ts, tt, true, part0, part1, &S->ticket)) return;
    const Z sts = sum_partials(part0, gridDim.x);
    const Z stt = sum_partials(part1, gridDim.x);
    if (threadIdx.x == 0) {
        S->ticket = 0;
        S->omega = stt.re == 0.0 ? Z{0.0, 0.0} : zdiv(sts, stt);
    }
}

__global__ void __launch_bounds__(kDotThreads) update_x_kernel(int n, const Z *y, const Z *z, const Z *s,
                                                               const Z *t, const Z *rh, Z *x, Z *r, Z *part0,
                                                               Z *part1, Scal *S) {
    if (S->stop) return;
    const Z alpha = S->alpha, omega = S->omega;
    Z rr = {0.0, 0.0}, hr = {0.0, 0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        x[i] = zadd(x[i], zadd(zmul(alpha, y[i]), zmul(omega, z[i])));
        const Z ri = zsub(s[i], zmul(omega, t[i]));
        r[i] = ri;
        rr = zadd(rr, zcdot(ri, ri));
        hr = zadd(hr, zcdot(rh[i], ri));
    }
    if (!partial_and_ticket(rr, hr, true, part0, part1, &S->ticket)) return;
    const Z srr = sum_partials(part0, gridDim.x);
    const Z rho = sum_partials(part1, gridDim.x);
    if (threadIdx.x == 0) {
        S->ticket = 0;
        S->rnorm2 = srr.re;
        S->iter += 1;
        if (S->rnorm2 <= S->tol2 * S->bnorm2) {
            S->stop = 1;
        } else if ((omega.re == 0.0 && omega.im == 0.0) || (rho.re == 0.0 && rho.im == 0.0)) {
            S->stop = 2;
        } else {
            S->beta = zmul(zdiv(rho, S->rho), zdiv(alpha, omega));
            S->rho = rho;
        }
    }
}

__global__ void scatter_u_kernel(const int32_t *unk, int nu, const Z *x, double *u) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nu) return;
    u[2 * unk[r]] = x[r].re;
    u[2 * unk[r] + 1] = x[r].im;
}

__global__ void residual_kernel(const Z *Kx, const Z *b, int n, Z *res) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) res[i] = zsub(b[i], Kx[i]);
}

sdd_status rb_arg(const char *msg) { return (sdd_status)report_error(SDD_E_ARG, msg); }
sdd_status rb_cuda(cudaError_t e, const char *what) {
    return (sdd_status)report_error(SDD_E_CUDA, (std::string(what) + ": " + cudaGetErrorString(e)).c_str());
}
#define RB_CUDA(call)                                                \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return rb_cuda(e_, #call);            \
    } while (0)

struct RbScratch {
    std::vector<void *> ptrs;
    cudaStream_t st = nullptr;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    ~RbScratch() {
        for (void *p : ptrs) cudaFree(p);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        if (st) cudaStreamDestroy(st);
    }
    template <class T>
    cudaError_t alloc(T **p, size_t count) {
        cudaError_t e = cudaMalloc((void **)p, (count ? count : 1) * sizeof(T));
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
};

sdd_status check_nodes_eps(const double *nodes_xz, int32_t n, int32_t ns, double eps) {
    if (ns < 2 || ns > kMaxStencil) return rb_arg("n_stencil must be in 2 .. SDD_RBFFD_MAX_STENCIL");
    if (n < ns || n > SDD_RBFFD_MAX_NODES) return rb_arg("n must be in n_stencil .. SDD_RBFFD_MAX_NODES");
    if (!(eps > 0.0) || !std::isfinite(eps)) return rb_arg("eps must be finite and > 0");
    if (!nodes_xz) return rb_arg("nodes_xz must not be NULL");
    for (int i = 0; i < 2 * n; ++i)
        if (!std::isfinite(nodes_xz[i])) return rb_arg("nodes must be finite");
    return SDD_OK;
}

// Stencils and weights on the device (d_p: nodes), timed by ev[0..2].
sdd_status weights_device(const double *h_p, const double *d_p, int n, int ns, double eps, int32_t *d_st,
                          double *d_w, RbScratch &S) {
    // the cell grid: about 2 nodes per cell over the bounding box, at most
    // 4 n + 16 cells
    double x0 = h_p[0], x1 = h_p[0], z0 = h_p[1], z1 = h_p[1];
    for (int i = 1; i < n; ++i) {
        x0 = std::min(x0, h_p[2 * i]);
        x1 = std::max(x1, h_p[2 * i]);
        z0 = std::min(z0, h_p[2 * i + 1]);
        z1 = std::max(z1, h_p[2 * i + 1]);
    }
    const double W = x1 - x0, H = z1 - z0, L = std::max(W, H);
    CellGrid g;
    g.x0 = x0;
    g.z0 = z0;
    g.c = W > 0.0 && H > 0.0 ? std::sqrt(2.0 * W * H / n) : (L > 0.0 ? 2.0 * L / n : 1.0);
    for (;;) {
        const double gx = std::floor(W / g.c) + 1.0, gz = std::floor(H / g.c) + 1.0;
        if (gx * gz <= 4.0 * n + 16.0) {
            g.gx = (int)gx;
            g.gz = (int)gz;
            break;
        }
        g.c *= 1.5;
    }
    const int m = g.gx * g.gz;
    int *d_err;
    int32_t *d_cell, *d_count, *d_start, *d_cursor, *d_list;
    RB_CUDA(S.alloc(&d_err, 1));
    RB_CUDA(S.alloc(&d_cell, (size_t)n));
    RB_CUDA(S.alloc(&d_count, (size_t)m));
    RB_CUDA(S.alloc(&d_start, (size_t)m + 1));
    RB_CUDA(S.alloc(&d_cursor, (size_t)m));
    RB_CUDA(S.alloc(&d_list, (size_t)n));
    RB_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), S.st));
    RB_CUDA(cudaMemsetAsync(d_count, 0, (size_t)m * sizeof(int32_t), S.st));
    RB_CUDA(cudaEventRecord(S.ev[0], S.st));
    cell_count_kernel<<<(n + 127) / 128, 128, 0, S.st>>>(d_p, n, g, d_cell, d_count);
    cell_scan_kernel<<<1, 1024, 0, S.st>>>(d_count, m, d_start);
    RB_CUDA(cudaMemcpyAsync(d_cursor, d_start, (size_t)m * sizeof(int32_t), cudaMemcpyDeviceToDevice, S.st));
    cell_fill_kernel<<<(n + 127) / 128, 128, 0, S.st>>>(d_cell, n, d_cursor, d_list);
    knn_kernel<<<(n + 127) / 128, 128, 0, S.st>>>(d_p, n, ns, g, d_start, d_list, d_st);
    RB_CUDA(cudaGetLastError());
    RB_CUDA(cudaEventRecord(S.ev[1], S.st));
    weights_kernel<<<(n + 63) / 64, 64, 0, S.st>>>(d_p, n, d_st, ns, eps, d_w, d_err);
    RB_CUDA(cudaGetLastError());
    RB_CUDA(cudaEventRecord(S.ev[2], S.st));
    int h_err = 0;
    RB_CUDA(cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, S.st));
    RB_CUDA(cudaStreamSynchronize(S.st));
    if (h_err) return rb_arg("a stencil matrix is singular (coincident nodes)");
    return SDD_OK;
}

}  // namespace
}  // namespace sdd

using namespace sdd;

extern "C" sdd_status sdd_rbffd_weights(const double *nodes_xz, int32_t n, int32_t n_stencil, double eps,
                                        int32_t *stencil, double *weights) {
    sdd_status r = check_nodes_eps(nodes_xz, n, n_stencil, eps);
    if (r != SDD_OK) return r;
    if (!stencil || !weights) return rb_arg("stencil and weights must not be NULL");
    RbScratch S;
    double *d_p, *d_w;
    int32_t *d_st;
    RB_CUDA(S.alloc(&d_p, 2 * (size_t)n));
    RB_CUDA(S.alloc(&d_st, (size_t)n * n_stencil));
    RB_CUDA(S.alloc(&d_w, (size_t)n * n_stencil));
    RB_CUDA(cudaStreamCreateWithFlags(&S.st, cudaStreamNonBlocking));
    for (int k = 0; k < 3; ++k) RB_CUDA(cudaEventCreate(&S.ev[k]));
    RB_CUDA(cudaMemcpyAsync(d_p, nodes_xz, 2 * (size_t)n * sizeof(double), cudaMemcpyHostToDevice, S.st));
    r = weights_device(nodes_xz, d_p, n, n_stencil, eps, d_st, d_w, S);
    if (r != SDD_OK) return r;
    RB_CUDA(cudaMemcpyAsync(stencil, d_st, (size_t)n * n_stencil * sizeof(int32_t), cudaMemcpyDeviceToHost, S.st));
    RB_CUDA(cudaMemcpyAsync(weights, d_w, (size_t)n * n_stencil * sizeof(double), cudaMemcpyDeviceToHost, S.st));
    RB_CUDA(cudaStreamSynchronize(S.st));
    return SDD_OK;
}

extern "C" sdd_status sdd_rbffd_solve(const double *nodes_xz, int32_t n, const uint8_t *dirichlet,
                                      const double *values, const double *kappa, int32_t n_stencil,
                                      double eps, double tol, int32_t max_iter, double *u,
                                      sdd_rbffd_stats *stats) {
    if (stats) *stats = sdd_rbffd_stats{};
    sdd_status r = check_nodes_eps(nodes_xz, n, n_stencil, eps);
    if (r != SDD_OK) return r;
    if (!dirichlet || !values || !kappa || !u) return rb_arg("dirichlet, values, kappa and u must not be NULL");
    if (!(tol > 0.0) || !std::isfinite(tol)) return rb_arg("tol must be finite and > 0");
    if (max_iter < 1) return rb_arg("max_iter must be at least 1");
    std::vector<int32_t> unk, pos(n, -1);
    for (int i = 0; i < n; ++i) {
        if (dirichlet[i] > 1) return rb_arg("dirichlet flags must be 0 or 1");
        if (!std::isfinite(kappa[i])) return rb_arg("kappa must be finite");
        if (dirichlet[i]) {
            if (!std::isfinite(values[2 * i]) || !std::isfinite(values[2 * i + 1]))
                return rb_arg("Dirichlet values must be finite");
        } else {
            pos[i] = (int32_t)unk.size();
            unk.push_back(i);
        }
    }
    const int nu = (int)unk.size();
    for (int i = 0; i < n; ++i) {
        u[2 * i] = dirichlet[i] ? values[2 * i] : 0.0;
        u[2 * i + 1] = dirichlet[i] ? values[2 * i + 1] : 0.0;
    }
    if (stats) stats->unknowns = nu;
    if (nu == 0) return SDD_OK;

    const int ns = n_stencil;
    RbScratch S;
    double *d_p, *d_w, *d_vals, *d_kap, *d_ew, *d_u;
    int32_t *d_st, *d_unk, *d_pos, *d_ecol;
    Z *d_dinv, *d_b, *x, *rr, *rh, *p, *v, *y, *s, *zz, *t, *part0, *part1;
    Scal *d_S;
    RB_CUDA(S.alloc(&d_p, 2 * (size_t)n));
    RB_CUDA(S.alloc(&d_st, (size_t)n * ns));
    RB_CUDA(S.alloc(&d_w, (size_t)n * ns));
    RB_CUDA(S.alloc(&d_vals, 2 * (size_t)n));
    RB_CUDA(S.alloc(&d_kap, (size_t)n));
    RB_CUDA(S.alloc(&d_unk, (size_t)nu));
    RB_CUDA(S.alloc(&d_pos, (size_t)n));
    RB_CUDA(S.alloc(&d_ew, (size_t)nu * ns));
    RB_CUDA(S.alloc(&d_ecol, (size_t)nu * ns));
    RB_CUDA(S.alloc(&d_u, 2 * (size_t)n));
    for (Z **q : {&d_dinv, &d_b, &x, &rr, &rh, &p, &v, &y, &s, &zz, &t}) RB_CUDA(S.alloc(q, (size_t)nu));
    RB_CUDA(S.alloc(&part0, (size_t)kDotBlocks));
    RB_CUDA(S.alloc(&part1, (size_t)kDotBlocks));
    RB_CUDA(S.alloc(&d_S, 1));
    RB_CUDA(cudaStreamCreateWithFlags(&S.st, cudaStreamNonBlocking));
    for (int k = 0; k < 5; ++k) RB_CUDA(cudaEventCreate(&S.ev[k]));
    cudaStream_t st = S.st;
    RB_CUDA(cudaMemcpyAsync(d_p, nodes_xz, 2 * (size_t)n * sizeof(double), cudaMemcpyHostToDevice, st));
    RB_CUDA(cudaMemcpyAsync(d_vals, u, 2 * (size_t)n * sizeof(double), cudaMemcpyHostToDevice, st));
    RB_CUDA(cudaMemcpyAsync(d_kap, kappa, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, st));
    RB_CUDA(cudaMemcpyAsync(d_unk, unk.data(), (size_t)nu * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    RB_CUDA(cudaMemcpyAsync(d_pos, pos.data(), (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    r = weights_device(nodes_xz, d_p, n, ns, eps, d_st, d_w, S);
    if (r != SDD_OK) return r;

    const int gb = (nu + 127) / 128;
    const int gd = std::min(kDotBlocks, (nu + kDotThreads - 1) / kDotThreads);
    assemble_kernel<<<gb, 128, 0, st>>>(d_unk, d_pos, nu, d_st, d_w, ns, d_kap, d_vals, d_ew, d_ecol, d_dinv, d_b);
    RB_CUDA(cudaGetLastError());
    // x = 0, r = r^ = b, p = v = 0
    RB_CUDA(cudaMemsetAsync(x, 0, (size_t)nu * sizeof(Z), st));
    RB_CUDA(cudaMemsetAsync(p, 0, (size_t)nu * sizeof(Z), st));
    RB_CUDA(cudaMemsetAsync(v, 0, (size_t)nu * sizeof(Z), st));
    RB_CUDA(cudaMemcpyAsync(rr, d_b, (size_t)nu * sizeof(Z), cudaMemcpyDeviceToDevice, st));
    RB_CUDA(cudaMemcpyAsync(rh, d_b, (size_t)nu * sizeof(Z), cudaMemcpyDeviceToDevice, st));
    dot_partial_kernel<<<gd, kDotThreads, 0, st>>>(d_b, d_b, nullptr, nu, part0, nullptr);
    RB_CUDA(cudaGetLastError());
    std::vector<Z> h_part(gd);
    RB_CUDA(cudaMemcpyAsync(h_part.data(), part0, gd * sizeof(Z), cudaMemcpyDeviceToHost, st));
    RB_CUDA(cudaStreamSynchronize(st));
    double bnorm2 = 0.0;
    for (int k = 0; k < gd; ++k) bnorm2 += h_part[k].re;
    Scal h_S{};
    h_S.alpha = h_S.omega = Z{1.0, 0.0};
    h_S.beta = Z{0.0, 0.0};
    h_S.rho = Z{bnorm2, 0.0};  // <r^, r> with r^ = r = b
    h_S.bnorm2 = bnorm2;
    h_S.rnorm2 = bnorm2;
    h_S.tol2 = tol * tol;
    if (bnorm2 == 0.0) h_S.stop = 1;  // zero right-hand side: x = 0
    RB_CUDA(cudaMemcpyAsync(d_S, &h_S, sizeof(Scal), cudaMemcpyHostToDevice, st));
    RB_CUDA(cudaEventRecord(S.ev[3], st));

    // iterations in batches of kPoll, replayed as one CUDA graph; the host
    // reads the scalars after each batch
    const int gi = std::min(kDotBlocks, (nu + kDotThreads - 1) / kDotThreads);
    auto iteration = [&]() {
        update_p_kernel<<<gi, kDotThreads, 0, st>>>(nu, d_S, rr, v, d_dinv, p, y);
        spmv_alpha_kernel<<<gi, kDotThreads, 0, st>>>(d_ew, d_ecol, nu, ns, d_unk, d_kap, y, rh, v, part0, d_S);
        update_s_kernel<<<gi, kDotThreads, 0, st>>>(nu, d_S, rr, v, d_dinv, s, zz);
        spmv_omega_kernel<<<gi, kDotThreads, 0, st>>>(d_ew, d_ecol, nu, ns, d_unk, d_kap, zz, s, t, part0, part1,
                                                      d_S);
        update_x_kernel<<<gi, kDotThreads, 0, st>>>(nu, y, zz, s, t, rh, x, rr, part0, part1, d_S);
    };
    const int kPoll = 8;
    cudaGraphExec_t gexec = nullptr;
    if (max_iter >= kPoll && !h_S.stop) {
        cudaGraph_t graph;
        RB_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        for (int q = 0; q < kPoll; ++q) iteration();
        RB_CUDA(cudaStreamEndCapture(st, &graph));
        const cudaError_t e = cudaGraphInstantiate(&gexec, graph, 0);
        cudaGraphDestroy(graph);
        RB_CUDA(e);
    }
    struct GraphGuard {
        cudaGraphExec_t g;
        ~GraphGuard() {
            if (g) cudaGraphExecDestroy(g);
        }
    } gguard{gexec};
    int it = 0;
    while (it < max_iter && !h_S.stop) {
        const int batch = std::min(kPoll, max_iter - it);
        if (batch == kPoll && gexec) {
            RB_CUDA(cudaGraphLaunch(gexec, st));
        } else {
            for (int q = 0; q < batch; ++q) iteration();
            RB_CUDA(cudaGetLastError());
        }
        RB_CUDA(cudaMemcpyAsync(&h_S, d_S, sizeof(Scal), cudaMemcpyDeviceToHost, st));
        RB_CUDA(cudaStreamSynchronize(st));
        it += batch;
    }
    // the true residual |b - K x| / |b|
    spmv_kernel<<<gb, 128, 0, st>>>(d_ew, d_ecol, nu, ns, d_unk, d_kap, x, t);
    residual_kernel<<<gb, 128, 0, st>>>(t, d_b, nu, s);
    dot_partial_kernel<<<gd, kDotThreads, 0, st>>>(s, s, nullptr, nu, part0, nullptr);
    RB_CUDA(cudaGetLastError());
    RB_CUDA(cudaMemcpyAsync(d_u, u, 2 * (size_t)n * sizeof(double), cudaMemcpyHostToDevice, st));
    scatter_u_kernel<<<gb, 128, 0, st>>>(d_unk, nu, x, d_u);
    RB_CUDA(cudaGetLastError());
    RB_CUDA(cudaMemcpyAsync(u, d_u, 2 * (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, st));
    RB_CUDA(cudaMemcpyAsync(h_part.data(), part0, gd * sizeof(Z), cudaMemcpyDeviceToHost, st));
    RB_CUDA(cudaEventRecord(S.ev[4], st));
    RB_CUDA(cudaStreamSynchronize(st));
    double res2 = 0.0;
    for (int k = 0; k < gd; ++k) res2 += h_part[k].re;
    if (stats) {
        float ms = 0.f;
        stats->iterations = h_S.iter;
        stats->rel_residual = bnorm2 > 0.0 ? std::sqrt(res2 / bnorm2) : 0.0;
        RB_CUDA(cudaEventElapsedTime(&ms, S.ev[0], S.ev[1]));
        stats->knn_ms = ms;
        RB_CUDA(cudaEventElapsedTime(&ms, S.ev[1], S.ev[2]));
        stats->weights_ms = ms;
        RB_CUDA(cudaEventElapsedTime(&ms, S.ev[3], S.ev[4]));
        stats->solve_ms = ms;
    }
    if (h_S.stop == 2) return (sdd_status)report_error(SDD_E_TIMEOUT, "BiCGStab broke down before convergence");
    if (h_S.stop != 1) return (sdd_status)report_error(SDD_E_TIMEOUT, "BiCGStab did not reach tol within max_iter");
    return SDD_OK;
}
