// Double-precision walk (the parity mode).
//
// Every quantity of the walk is FP64 and every discrete decision (exit on
// overshoot, bridge hit, material of a point, counts) is taken with the
// expressions of their definitions in absolute coordinates, so that on the
// same Philox streams the walks agree path by path with any other FP64
// implementation of the same definitions, up to the last-ulp differences of
// log/sin/cos.  Compiled with -fmad=false: no product is fused into a sum.
//
// Steps (Sec. 3.1): uniforms (w + 1/2) 2^-32; W = sqrt(-2 ln u0)
// (cos 2 pi u1, sin 2 pi u1); beta' = beta + sqrt(dt) W; overshoot ->
// theta = d / (d - d') (first-exit-time estimate, second case); both inside
// -> hit iff min_w 2 d_w d'_w / dt <= -ln U (first case with kappa_i = 1);
// else the step counts for the material of beta'.
#include "walk_sched.cuh"
#include "walk_tm.cuh"

namespace sdd {

__device__ __forceinline__ double uni32(uint32_t w) {
    return ((double)w + 0.5) * (1.0 / 4294967296.0);
}

template <int KMAX_, int GEO>
struct WalkerF64 {
    using Real = double;
    static constexpr int KMAX = KMAX_;
    static constexpr bool kCoop = false;  // no cooperative tail: the parity walk stays plain
    static constexpr bool kGrouped = false;  // one queue (a grouped plan's order is one queue too)
    static constexpr int kMinCTAs = 3;
    using Occ = uint32_t;
    using HistT = uint32_t;
    static constexpr int kStored = KMAX - 1;
    static constexpr int kHist = 1;

    double x, z;
    uint32_t n;
    uint32_t cnt[KMAX > 1 ? KMAX - 1 : 1];
    int mcur;
    uint32_t nid;

    __device__ static int material(const ModelDev &M, double x, double z) {
        if (GEO == GEO_RASTER) {
            const double fx = floor((x - M.xmin) * M.sx);
            const double fz = floor((z - M.zmin) * M.sz);
            long long ix = (long long)fx, iz = (long long)fz;
            if (ix < 0) ix = 0;
            if (ix > M.nx - 1) ix = M.nx - 1;
            if (iz < 0) iz = 0;
            if (iz > M.nz - 1) iz = M.nz - 1;
            return (int)__ldg(M.raster + iz * (long long)M.nx + ix);
        } else {
            int m = (z >= 0.0) ? M.bg_earth : M.bg_air;
            for (int s = 0; s < M.n_shapes; ++s) {
                const ShapeDev &S = M.shapes[s];
                const double *v = S.d;
                bool in;
                if (S.kind == 0) {
                    in = (x >= v[0] && x < v[1] && z >= v[2] && z < v[3]);
                } else {
                    const double sg = S.dsign;
                    const double e0 = sg * ((v[2] - v[0]) * (z - v[1]) - (v[3] - v[1]) * (x - v[0]));
                    const double e1 = sg * ((v[4] - v[2]) * (z - v[3]) - (v[5] - v[3]) * (x - v[2]));
                    const double e2 = sg * ((v[0] - v[4]) * (z - v[5]) - (v[1] - v[5]) * (x - v[4]));
                    in = (e0 >= 0.0 && e1 >= 0.0 && e2 >= 0.0);
                }
                if (in) m = S.mat;
            }
            return m;
        }
    }

    __device__ __forceinline__ void bind(HistT *) {}

    __device__ __forceinline__ void counts(const ModelDev &, uint32_t, uint32_t *c) const {
#pragma unroll
        for (int j = 0; j < (KMAX > 1 ? KMAX - 1 : 1); ++j) c[j] = cnt[j];
    }

    __device__ __forceinline__ void count(int m) {
#pragma unroll
        for (int j = 1; j < KMAX; ++j) cnt[j - 1] += (m == j) ? 1u : 0u;
    }

    __device__ __forceinline__ void start(const ModelDev &M, const WalkArgs &A, double x0,
                                          double z0, uint32_t path, uint32_t node_id, int) {
        x = x0;
        z = z0;
        n = 0;
#pragma unroll
        for (int j = 0; j < (KMAX > 1 ? KMAX - 1 : 1); ++j) cnt[j] = 0;
        mcur = material(M, x0, z0);
        nid = node_id;
    }

    __device__ static void place(const ModelDev &M, double x, double z, double xn, double zn,
                                 double th, int w, ExitInfo<double> &ei) {
        ei.th = th;
        ei.wall = w;
        ei.x = x + th * (xn - x);
        ei.z = z + th * (zn - z);
        if (w == 0) ei.x = M.xmin;
        if (w == 1) ei.x = M.xmax;
        if (w == 2) ei.z = M.zmin;
        if (w == 3) ei.z = M.zmax;
    }

    __device__ int substep(const ModelDev &M, const WalkArgs &A, uint32_t path, uint32_t wa,
                           uint32_t wb, ExitInfo<double> &ei) {
        const double u0 = uni32(wa), u1 = uni32(wb);
        const double rho = sqrt(-2.0 * log(u0));
        const double ang = 6.283185307179586 * u1;
        const double w0 = rho * cos(ang);
        const double w1 = rho * sin(ang);
        const double xn = x + A.sdt * w0;
        const double zn = z + A.sdt * w1;
        const double d[4] = {x - M.xmin, M.xmax - x, z - M.zmin, M.zmax - z};
        const double dn[4] = {xn - M.xmin, M.xmax - xn, zn - M.zmin, M.zmax - zn};
        if (dn[0] <= 0.0 || dn[1] <= 0.0 || dn[2] <= 0.0 || dn[3] <= 0.0) {
            double best = 2.0;
            int bw = 0;
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                if (dn[w] <= 0.0) {
                    const double t = d[w] / (d[w] - dn[w]);
                    if (t < best) { best = t; bw = w; }
                }
            }
            place(M, x, z, xn, zn, best, bw, ei);
            ei.mlast = mcur;
            ei.nocc = n;
            return 1;
        }
        double best = 2.0 * d[0] * dn[0] / A.dt;
        int bw = 0;
#pragma unroll
        for (int w = 1; w < 4; ++w) {
            const double e = 2.0 * d[w] * dn[w] / A.dt;
            if (e < best) { best = e; bw = w; }
        }
        // -ln U <= 33 ln 2 < 23 for U >= 2^-33: no uniform can hit above 23
        if (best <= 23.0) {
            const uint4 b = philox4x32_10(make_uint4(n, path, nid, 1u), A.key0, A.key1);
            const double L = -log(uni32(b.x));
            if (best <= L) {
                place(M, x, z, xn, zn, best / L, bw, ei);
                ei.mlast = mcur;
                ei.nocc = n;
                return 1;
            }
        }
        const int m = material(M, xn, zn);
        count(m);
        x = xn;
        z = zn;
        mcur = m;
        ++n;
        if (n >= A.max_steps) {
            ei.x = x; ei.z = z; ei.th = 0.0; ei.wall = 0;
            ei.mlast = mcur;
            ei.nocc = n;
            return 2;
        }
        return 0;
    }

    __device__ __forceinline__ int iterate(const ModelDev &M, const WalkArgs &A, uint32_t path,
                                           ExitInfo<double> &ei) {
        const uint4 w = philox4x32_10(make_uint4(n >> 1, path, nid, 0u), A.key0, A.key1);
        const int r = substep(M, A, path, w.x, w.y, ei);
        if (r) return r;
        return substep(M, A, path, w.z, w.w, ei);
    }

    __device__ static void to_abs(const ModelDev &, double X, double Z, double &ox, double &oz) {
        ox = X;
        oz = Z;
    }

    __device__ static double2 column(double kr, double ki, double z) {
        if (z >= 0.0) {
            const double a = exp(-kr * z);
            double s, c;
            sincos(ki * z, &s, &c);
            return make_double2(a * c, -a * s);
        }
        return make_double2(1.0 - kr * z, -(ki * z));
    }

    __device__ static double2 sample(const ModelDev &M, const SharedTables &T, const WalkArgs &A,
                                     int, int e, double x, double z, double th, int wall, int mlast,
                                     const uint32_t *c) {
        const double dt = A.dt;
        const double *kap = T.kappa + e * M.K;
        double ph = 0.0;
#pragma unroll
        for (int k = 0; k < KMAX; ++k)
            if (k < M.K) ph += kap[k] * ((double)c[k] * dt);
        ph += kap[mlast] * (th * dt);
        ph *= 0.5;
        double sw, cw;
        sincos(ph, &sw, &cw);
        double2 g;
        if (M.g_kind == 1) {
            const double *a = M.g_coef;
            g = make_double2(a[0] + a[2] * x + a[4] * z, a[1] + a[3] * x + a[5] * z);
        } else if (M.g_kind == 2) {
            g = make_double2(x * x - z * z, 0.0);
        } else {
            const EvalDev &E = T.ev[e];
            if (wall == 0) {
                g = column(E.kl_re, E.kl_im, z);
            } else if (wall == 1) {
                g = column(E.kr_re, E.kr_im, z);
            } else {
                const double t = (x - M.xmin) / (M.xmax - M.xmin);
                const double lr = wall == 2 ? E.tl_re : E.bl_re, li = wall == 2 ? E.tl_im : E.bl_im;
                const double rr = wall == 2 ? E.tr_re : E.br_re, ri = wall == 2 ? E.tr_im : E.br_im;
                g = make_double2((1.0 - t) * lr + t * rr, (1.0 - t) * li + t * ri);
            }
        }
        // (cw - i sw)(g.x + i g.y)
        return make_double2(cw * g.x + sw * g.y, cw * g.y - sw * g.x);
    }
};

template <int KMAX, int GEO>
static cudaError_t launch_one(const ModelDev &M, const WalkArgs &A, int grid, int block,
                              cudaStream_t s) {
    const size_t sm = shared_bytes<WalkerF64<KMAX, GEO>>(block / 32, M.E, M.K);
    auto k = walk_kernel<WalkerF64<KMAX, GEO>>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k<<<grid, block, sm, s>>>(M, A);
    return cudaGetLastError();
}

template <int KMAX, int GEO>
static int occ_one(int block, int E, int K) {
    const size_t sm = shared_bytes<WalkerF64<KMAX, GEO>>(block / 32, E, K);
    auto k = walk_kernel<WalkerF64<KMAX, GEO>>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, block, sm) != cudaSuccess) return 0;
    return n;
}

#define SDD_DISPATCH(FN, ...)                                                   \
    switch (kmax * 2 + geo) {                                                   \
    case 4: return FN<2, GEO_SHAPES>(__VA_ARGS__);                              \
    case 5: return FN<2, GEO_RASTER>(__VA_ARGS__);                              \
    case 6: return FN<3, GEO_SHAPES>(__VA_ARGS__);                              \
    case 7: return FN<3, GEO_RASTER>(__VA_ARGS__);                              \
    case 8: return FN<4, GEO_SHAPES>(__VA_ARGS__);                              \
    case 9: return FN<4, GEO_RASTER>(__VA_ARGS__);                              \
    case 16: return FN<8, GEO_SHAPES>(__VA_ARGS__);                             \
    case 17: return FN<8, GEO_RASTER>(__VA_ARGS__);                             \
    default: break;                                                             \
    }

// The TM parity walk (vertical strips).
template <int KMAX>
static cudaError_t launch_tm(const ModelDev &M, const WalkArgs &A, int grid, int block, cudaStream_t s) {
    using W = WalkerTM<double, KMAX>;
    const size_t sm = shared_bytes<W>(block / 32, M.E, M.K);
    auto k = walk_kernel<W>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k<<<grid, block, sm, s>>>(M, A);
    return cudaGetLastError();
}

template <int KMAX>
static int occ_tm(int block, int E, int K) {
    using W = WalkerTM<double, KMAX>;
    const size_t sm = shared_bytes<W>(block / 32, E, K);
    auto k = walk_kernel<W>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, block, sm) != cudaSuccess) return 0;
    return n;
}

#define SDD_TM_DISPATCH(FN, ...)                                                \
    switch (kmax) {                                                             \
    case 2: return FN<2>(__VA_ARGS__);                                          \
    case 3: return FN<3>(__VA_ARGS__);                                          \
    case 4: return FN<4>(__VA_ARGS__);                                          \
    case 8: return FN<8>(__VA_ARGS__);                                          \
    default: break;                                                             \
    }

cudaError_t launch_walk_f64(int kmax, int geo, const ModelDev &M, const WalkArgs &A, int grid,
                            int block, cudaStream_t s) {
    if (geo == GEO_TM) {
        SDD_TM_DISPATCH(launch_tm, M, A, grid, block, s)
        return cudaErrorInvalidValue;
    }
    SDD_DISPATCH(launch_one, M, A, grid, block, s)
    return cudaErrorInvalidValue;
}

int occupancy_f64(int kmax, int geo, int block, int E, int K) {
    if (geo == GEO_TM) {
        SDD_TM_DISPATCH(occ_tm, block, E, K)
        return 0;
    }
    SDD_DISPATCH(occ_one, block, E, K)
    return 0;
}

}  // namespace sdd
