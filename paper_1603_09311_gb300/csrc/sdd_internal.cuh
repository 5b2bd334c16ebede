// Internal device-side definitions of libsdd (not part of the C ABI).
//
// Shared by the host API (sdd_api.cu) and the two walk translation units
// (walk_f32.cu: single-precision walk; walk_f64.cu: double-precision parity
// walk compiled without FMA contraction).
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

struct sdd_ctx;

namespace sdd {

constexpr int kMaxK = 8;
constexpr int kMaxE = 32;
constexpr int kMaxShapes = 16;
constexpr int kRing = 64;  // exit records buffered per warp

enum Geo : int { GEO_SHAPES = 0, GEO_RASTER = 1, GEO_TM = 2 };

// Material-lookup programs of the single-precision walk, chosen per model so
// that the common cases run without loops or branches: the layered
// background alone, exactly one rectangle, exactly one triangle, up to 4 or
// up to 16 shapes (unrolled, guarded), or the int8 raster.
// GC_CONTACT is one rectangle [x0, >= x_max) x [0, >= z_max): the earth split
// by a vertical contact at x0 (the quarter-space model), tested with two
// compares; it takes the same decisions as GC_RECT1 on every inside point.
// GC_RECT1 is one rectangle wholly on one side of the surface z = 0.  These
// two programs count steps by region (earth side, inside the shape) rather
// than by material, and turn the region counts into material counts at the
// walk's exit.
// GC_RASTER_MULTI serves a batch of raster models sharing the domain and the
// raster size: each lane reads the raster of its walk's model.  GC_TM is the
// TM walk over vertical strips (its own walker).
enum GeoCode : int { GC_LAYER = 0, GC_RECT1 = 1, GC_TRI1 = 2, GC_SHAPES4 = 3, GC_SHAPES16 = 4,
                     GC_RASTER = 5, GC_CONTACT = 6, GC_RASTER_MULTI = 7, GC_TM = 8 };



// One work item: paths [path0, path0 + count) of node `node` of model
// `model` (the index into WalkArgs::models of a batched launch, else 0).
struct Item {
    int32_t node;
    uint32_t path0;
    int32_t count;
    int32_t model;
};

// A material shape.  f: single-precision copy in domain-centred coordinates
// (rectangle bounds, or the three edge lines A X + B Z + C >= 0 of a
// triangle, orientation folded in).  d: double-precision absolute copy
// (rectangle bounds or the vertices), evaluated exactly as the definition.
struct ShapeDev {
    int32_t kind, mat;
    float f[9];
    double d[6];
    double dsign;  // orientation sign of a triangle
};

// Per-evaluation constants of the boundary data (SDD_G_COLUMNS): the column
// wavenumbers k = sqrt(i kappa) of the left and right columns and the four
// corner values used by the top/bottom interpolation.
struct EvalDev {
    double kl_re, kl_im, kr_re, kr_im;
    double tl_re, tl_im, tr_re, tr_im;  // top-left, top-right corners
    double bl_re, bl_im, br_re, br_im;  // bottom-left, bottom-right corners
};

constexpr int kMaxBatchModels = 256;

// Two-level form of an int8 raster, identical cell by cell: tiles of
// kTile x kTile cells; coarse[tz][tx] = kTileUniform | material for a tile of
// one material, else the index of the tile's kTile^2 cells in the pool.  The
// tiles start one tile before the raster and end at least one tile after it,
// their cells outside the raster repeating its nearest edge cell, so a cell
// index that rounding puts one past an edge needs no clamp.
constexpr int kTileShift = 4;
constexpr int kTile = 1 << kTileShift;
constexpr uint32_t kTileUniform = 0x80000000u;
__host__ __device__ constexpr int tile_cols(int n) { return n / kTile + 2; }
// Raster side limit: cell indices are formed by FP32 magic-number rounding,
// exact below 2^22.
constexpr int kMaxRasterSide = 1 << 20;

// Per-model data of a batched launch (device memory).
struct BatchModel {
    const int8_t *raster;
    const uint32_t *tcoarse;
    const uint8_t *tpool;
    int32_t K, pad;
    double kappa[kMaxE * kMaxK];  // [E][K] of this model
    EvalDev ev[kMaxE];
};

struct ModelDev {
    double xmin, xmax, zmin, zmax;
    double xc, zc, hw, hh;  // centre and half sizes
    int32_t K, E, Epad;
    int32_t bg_air, bg_earth;
    int32_t n_shapes;
    int32_t gcode;  // GeoCode of the model
    ShapeDev shapes[kMaxShapes];
    const int8_t *raster;
    const uint32_t *tcoarse;  // two-level form of the raster (single-precision walk)
    const uint8_t *tpool;
    int32_t ntx;              // tiles per raster row
    uint32_t tpool_off;       // bytes from the coarse table to the pool (same for every model
                              // of a batch: the coarse table rounded up to 256 bytes)
    int32_t nx, nz;
    double sx, sz;  // nx / (xmax - xmin), nz / (zmax - zmin)
    int32_t g_kind;
    double g_coef[6];
    double kappa[kMaxE * kMaxK];  // [E][K]
    EvalDev ev[kMaxE];
    // single-precision constants of the centred walk (X = x - xc, Z = z - zc)
    float fhw, fhh;  // half width / height
    float fxc, fzc;  // centre
    float fzs;       // earth surface z = 0 in centred coordinates
    float fsx, fsz;  // raster cells per unit length
    float fox, foz;  // hw * sx - 1/2 + kTile, hh * sz - 1/2 + kTile: round(X sx + ox) is the
                     // cell index plus kTile (the tile map's margin)
    // GC_RECT1 / GC_CONTACT: 1 when the one shape lies wholly in the air
    // (z < 0), 0 when wholly in the earth; a shape that straddles the
    // surface is served by GC_SHAPES4 instead
    int32_t shape_air;
    // TM mode: material m is the vertical strip [xif[m-1], xif[m]) with
    // diffusion diff[m]
    int32_t tm;
    double diff[kMaxK], xif[kMaxK];
    float fdiff[kMaxK], fxif[kMaxK];
    double tm_a[kMaxE][kMaxK][2];  // boundary data kind 3: sqrt(i kappa_{e,m} / D_m)
};

struct WalkArgs {
    const Item *items;
    int32_t n_items;
    const int32_t *order;      // [n_items] item of each queue position (nullptr: identity)
    const double *nodes;       // [n][2] absolute
    const uint32_t *node_ids;  // nullable
    double dt;
    double sdt;                // sqrt(dt)
    float f_cdt;               // -2 ln(2) dt: squared step radius = f_cdt * log2(u0)
    float f_c2dt;              // 2 / dt
    float f_bthr;              // bridge filter: d d' above this cannot hit (single precision)
    uint32_t key0, key1;       // Philox key (seed)
    uint32_t rk0[10], rk1[10]; // the key of each Philox round (key bumped by the Weyl constants)
    uint32_t max_steps;
    double *slots;             // [n_items][E][4]: sum re, sum im, sum re^2, sum im^2
                               // (cleared by the warp that opens the item)
    int32_t *item_trunc;       // [n_items] truncated walks (cleared likewise)
    unsigned long long *counters;  // steps, walks, truncated
    int32_t *queue;            // next item (zero before launch); one counter per queue
    // grouped launches (several models): queue m hands out order[qbase[m] ..
    // qbase[m+1]); a CTA starts on queue m when (blockIdx + 1/2) / gridDim
    // falls in [home_cut[m], home_cut[m+1]) and moves on when it is empty
    const int32_t *qbase;      // [n_queues + 1] (nullptr: one queue over order)
    const float *home_cut;     // [n_queues + 1]
    int32_t n_queues;
    int32_t *error;            // nonzero if a device-side check failed
    const int32_t *cancel;     // nullable; nonzero: hand out no more paths (asynchronous requests)
    // per-path dump (sdd_walk_records); when rec_steps != nullptr the walk
    // records are written here instead of being summed
    int64_t *rec_steps;
    int64_t *rec_counts;       // [count][K] (nullable)
    double *rec_occ;           // [count][K] occupation in units of dt (nullable)
    int64_t *rec_hits;         // [count] interface randomisations (nullable)
    double *rec_exit;          // [count][3]
    int32_t *rec_wall;
    int32_t *rec_mlast;
    const BatchModel *models;  // batched launch: the models the items refer to
};

// Two-level tile map of an int8 raster [nz][nx] (host): coarse table
// [ceil(nz/kTile)][ceil(nx/kTile)] and pool of mixed tiles (cells beyond the
// raster edge repeat the nearest edge cell).
void build_tiles(const int8_t *raster, int nx, int nz, std::vector<uint32_t> &coarse,
                 std::vector<uint8_t> &pool);

// Launchers (one per precision translation unit).
cudaError_t launch_walk_f32(int kmax, int geo, const ModelDev &M, const WalkArgs &A, int grid,
                            int block, cudaStream_t s);
cudaError_t launch_walk_f64(int kmax, int geo, const ModelDev &M, const WalkArgs &A, int grid,
                            int block, cudaStream_t s);
// Record msg as the calling thread's last error (sdd_last_error) and return
// status.
int report_error(int status, const char *msg);

// TM models: *D = the diffusion of the strip holding x ([x_{m-1}, x_m)), 1
// returned; TE models: 0.
int ctx_site_diffusion(const ::sdd_ctx *c, double x, double *D);

// Largest number of resident CTAs per SM for a configuration.
int occupancy_f32(int kmax, int gcode, int block, int E, int K);
int occupancy_f64(int kmax, int geo, int block, int E, int K);
size_t smem_bytes(bool f64, int kmax, int block);

}  // namespace sdd
