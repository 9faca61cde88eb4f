/*
 * softshadow.h -- C ABI of the GB300 soft-shadow library (libsoftshadow.so).
 *
 * Soft shadows on a heightfield draped on a sphere, after Jung, Schrempp & Son,
 * "Optimally Fast Soft Shadows on Curved Terrain with Dynamic Programming and
 * Maximum Mipmaps" (arXiv 2005.06671).  For each surface point p one shadow ray
 * p + t*L is cast toward the centre of the sun (Sec. 3.1); its cost is the
 * clearance between the ray and the terrain divided by the distance travelled,
 * minimised over the ray (Eq. shadowfrac, final step of Algorithm 1); the
 * light fraction is the part of the sun disc left above the horizon chord that
 * cost implies (Eqs. discsegment/discfrac, Sec. 3.4).  The minimum is found by a
 * descent over a maximum mipmap (Sec. 3.2, "Dynamic Programming", "Maximum
 * mipmaps") made exact: every sample whose cost could beat the running minimum
 * is evaluated, so the result equals evaluating every sample.
 *
 * Conventions shared by every call
 * --------------------------------
 * Geometry.  Sphere of radius R centred at the origin.  Tile frame: x = grid +u
 * (columns), y = grid +v (rows), z = direction of the tile centre.  Texel (u, v)
 * (0-based column, row) sits at plane coordinates X = (u - (nx-1)/2)*g,
 * Y = (v - (ny-1)/2)*g, mapped to the sphere gnomonically (direction
 * (X, Y, R)/|.|; a straight 3-D ray maps to a straight texture line, Sec. 3.2,
 * Appendix "Deriving T") or by polar stereographic projection (tile centred on
 * the pole, projected from the antipode onto the plane z = R: direction
 * (4RX, 4RY, 4R^2 - X^2 - Y^2)/(4R^2 + X^2 + Y^2); a ray maps to a circular
 * arc).  ss_shadow_forward, ss_shadow_uniform and ss_shadow_backward take either
 * mapping; the batch calls take gnomonic tiles only (SS_ERR_UNSUPPORTED
 * otherwise).  Heights h are metres above the sphere.  Bilinear interpolation
 * uses base texel min(floor(u), nx-2); the usable domain is [0,nx-1]x[0,ny-1].
 * Sun direction s = (cos e sin a, cos e cos a, sin e) in the tile frame:
 * elevation e, azimuth a measured from grid +y toward grid +x.
 * Samples t_j = j * delta (j = 1 .. floor(max_len/delta)), delta = step_texels*g;
 * a sample is used when its texel image lies in the usable domain.
 *   cost c_j   = (|p + t_j s| - R - h(sample)) / t_j          [rad]
 *   c*         = min_j c_j, argmin j* = smallest j attaining it (1-based),
 *                or c* = +inf, j* = -1 when no sample is usable
 *   d          = clamp(c* cos(eps_p) / alpha, -1, 1), sin(eps_p) = n_p . s
 *   light      = (pi - acos d + d sqrt(1 - d^2)) / pi          (1 when j* = -1)
 *
 * Memory.  Every pointer named "device" is CUDA device memory owned by the
 * caller; the library never allocates device memory.  Heights are float32,
 * row-major, row stride pitch (elements).
 *
 * Non-finite inputs.  Heights, listed ray origins and lifts, and dL/dlight
 * should be finite.  A call never faults on non-finite ones (every texel index
 * is clamped to the tile), and reports them in the caller's device status word
 * when one is given (ss_outputs.status, the status argument of
 * ss_shadow_backward_ws): the word is OR-ed with SS_DEV_* bits, read it after
 * the stream has synchronised (zero it before the call).  Outputs: a ray
 * whose origin or lift is NaN has no usable sample (light 1, argmin -1); a
 * sample whose bilinear cell holds a NaN height has a NaN cost and is skipped,
 * as in the plain definition in IEEE arithmetic (NaN never compares below the
 * running minimum; maximum-mipmap levels ignore NaN texels).  Rays whose
 * origin cell holds a NaN (a grid ray takes its own texel's value), that
 * read an infinite height or start at an infinite origin get an unspecified
 * light in [0, 1] and argmin.  The non-finite height count comes from the
 * maximum-mipmap build of the same heights (its stats block), so it is
 * reported by the calls that take that mipmap.
 *
 * Streams.  Every call that takes an ss_stream_t enqueues its work on that
 * stream (NULL = the legacy default stream) and returns without synchronising.
 *
 * Errors.  Argument errors are detected on the host before anything is
 * enqueued and returned synchronously; CUDA launch errors map to SS_ERR_CUDA
 * (details: ss_last_error_string()).  Nothing is launched when a call fails
 * validation.
 */
#ifndef SOFTSHADOW_H
#define SOFTSHADOW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* ss_stream_t; /* a cudaStream_t */

typedef enum {
    SS_OK = 0,
    SS_ERR_INVALID_ARG = 1,   /* null pointer, non-finite or out-of-range scalar */
    SS_ERR_BAD_SIZE = 2,      /* nx/ny/pitch/ray count out of range            */
    SS_ERR_OUT_OF_MEMORY = 3, /* caller-supplied workspace too small            */
    SS_ERR_CUDA = 4,          /* a CUDA runtime call or launch failed           */
    SS_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up             */
    SS_ERR_INTERNAL = 6,      /* device-side consistency check failed           */
    SS_ERR_UNSUPPORTED = 7    /* valid request this build does not implement     */
} ss_status;

enum { SS_PROJ_GNOMONIC = 0, SS_PROJ_POLAR_STEREO = 1 };
enum { SS_RAYS_GRID = 0, SS_RAYS_LIST = 1 };

/* ss_params.flags */
#define SS_FLAG_COUNT_SAMPLES 0x1u /* fill ss_outputs.counters                      */
#define SS_FLAG_NO_EARLY_EXIT 0x2u /* ss_shadow_uniform: evaluate every usable sample */
/* Light-only mode (forward, uniform, batch).  The light depends on c* only
 * through clamp(c* cos(eps)/alpha, -1, 1) (Eq. discfrac), so the search may use
 * c_sat = 1.002 alpha / cos(eps): it starts from best = +c_sat (blocks whose
 * bound reaches it cannot change the light) and stops as soon as
 * best <= -c_sat (the ray is in full umbra).  light is exact as in the default
 * mode; argmin and cost are exact for rays in the penumbra; a fully lit ray
 * reports argmin -1, cost +inf; a ray in umbra reports the first sample found
 * with cost <= -c_sat (a witness, not necessarily the minimum). */
#define SS_FLAG_LIGHT_ONLY 0x4u

/* ss_shadow_backward_ws: deterministic accumulation (see there). */
#define SS_FLAG_DETERMINISTIC_BWD 0x8u
/* ss_shadow_forward, exact descent with column seeds (the default): a warp
 * evaluates the leaf samples its lanes' walks cannot prune as shared tasks, 32
 * at a time (the walks themselves only bound blocks); with this flag each lane
 * evaluates its own ray's leaf samples inside its walk.  Same results bit for
 * bit. */
#define SS_FLAG_LANE_LEAVES 0x10u

/* Bits of the device status word (ss_outputs.status, ss_shadow_backward_ws). */
#define SS_DEV_NONFINITE_HEIGHT 0x1u /* the heights hold a NaN or an infinity      */
#define SS_DEV_NONFINITE_RAY 0x2u    /* a listed origin or lift is NaN or infinite  */
#define SS_DEV_NONFINITE_GRAD 0x4u   /* a dL/dlight value is NaN or infinite (that
                                        ray contributes nothing)                    */

/* Largest supported tile edge and ray length (samples): sample indices and
 * texel coordinates are exact in float32 below these bounds. */
#define SS_MAX_DIM 65536
#define SS_MAX_SAMPLES 65535

/* Heightfield tile (Sec. 3.2: texture of heights draped on the sphere). */
typedef struct {
    const float* h;        /* device, [ny][pitch] float32 heights (m)          */
    int32_t nx, ny;        /* columns, rows; each in [2, SS_MAX_DIM]           */
    int64_t pitch;         /* row stride in elements, >= nx                    */
    double texel_m;        /* g: texel size on the projection plane (m), > 0   */
    double radius_m;       /* R: sphere radius (m), > 0                        */
    int32_t projection;    /* SS_PROJ_*                                        */
} ss_heightfield;

/* Light source: direction and angular radius r_L (Sec. 3.4). */
typedef struct {
    double elevation_rad;       /* e, in (-pi/2, pi/2)                         */
    double azimuth_rad;         /* a, from grid +y toward grid +x              */
    double angular_radius_rad;  /* alpha = r_L > 0                             */
} ss_sun;

typedef struct {
    double max_len_m;      /* Lmax: longest ray (m), > 0                       */
    double step_texels;    /* delta / g; 0 selects 0.5                         */
    uint32_t flags;        /* SS_FLAG_*                                        */
    int32_t block_threads; /* threads per block, multiple of 32 in [32, 256];
                              0 = 256                                          */
    int32_t leaf_level;    /* forward: subtrees of <= 2^leaf_level samples are
                              evaluated sample by sample; -1 = default (grid
                              rays and the batch 1, listed rays 2)             */
    int32_t rays_per_thread; /* forward kernels: a block owns block_threads x
                              rays_per_thread rays, in [0, 4096]; 0 = default
                              (descent: grid rays 24, listed rays 12; uniform
                              stepping 16)                                     */
    int32_t refill_min;    /* forward kernels: a warp's idle lanes take new
                              rays once at least this many are idle, in
                              [0, 32]; 0 = default (exact descent with leaf
                              tasks: 14 on gnomonic, 22 on stereographic
                              tiles; single-lane walks 10; else 6)             */
    int32_t ray_tile_w;    /* grid-mode rays: w > 0 = a block's rays form
                              rectangles of w x (rays / w) texels (w must
                              divide the block's or chunk's ray count);
                              0 = default: 256-wide rectangles for the exact
                              descent, runs of consecutive ray ids otherwise
                              (batch: a warp's chunk)                          */
    int32_t strip_len;     /* ss_shadow_forward and the batch (exact descent):
                              seeding of each ray's descent with the best of
                              its own samples next to a neighbouring ray's
                              argmin (a sample cost, an upper bound of the
                              minimum, so results are unchanged).  0 = default:
                              single rays drawn row by row, each seeded from
                              the last finished ray of its column (grid rays:
                              columns of the ray rectangle, at most 512 wide,
                              else strips of 10; listed rays: a block's ids
                              read as 512 columns of consecutive ids).
                              S in [2, 256]: each lane walks a strip of S
                              neighbouring rays (down a rectangle column, or
                              consecutive ids), seeding from the previous one.
                              In both seeded modes a ray with no finished
                              neighbour (a rectangle's first row, a strip's
                              first ray) is seeded with the best of its
                              samples j_lo - 1 + 2^k, k = 0, 1, ... and j_hi.
                              1 = no seeding.  Light-only forward: 0 as
                              above, any other value = no seeding.  Other
                              calls ignore it.                                 */
    int32_t seed_width;    /* seeded descents: a ray seeded from a neighbour's
                              argmin j evaluates its samples within +-w of
                              where j's terrain point lies along this ray
                              (grid rays; listed rays: of j itself), w in
                              [0, 16]; 0 = default (grid rays 1, listed
                              rays 2: neighbouring view rays can be several
                              texels apart)                                    */
} ss_params;

/* Ray origins p (Sec. 3.1: view-ray intersection points). */
typedef struct {
    int32_t mode;          /* SS_RAYS_GRID: one ray per texel centre, ray r at
                              (r % nx, r / nx), n = nx*ny;
                              SS_RAYS_LIST: n rays at uv[2r], uv[2r+1]        */
    int64_t n;             /* list mode: number of rays, >= 0                  */
    const float* uv;       /* device, [n][2] texel coordinates (list mode)     */
    const float* lift_m;   /* device, [n] metres above the surface, or NULL    */
} ss_rays;

/* Per-ray outputs, all device arrays of n entries. */
typedef struct {
    float* light;          /* required: lit fraction in [0, 1]                 */
    int32_t* argmin;       /* required: j* (1-based) or -1                     */
    float* cost;           /* optional: c* in rad (+inf when j* = -1), or NULL */
    int32_t* counters;     /* optional [n][2]: (bound probes, leaf samples)
                              when SS_FLAG_COUNT_SAMPLES is set, or NULL       */
    uint32_t* status;      /* optional device word OR-ed with SS_DEV_* bits
                              (non-finite heights or ray inputs), or NULL      */
} ss_outputs;

/* ---------------------------------------------------------------- general */
const char* ss_status_string(ss_status status);
/* Text of the last CUDA error seen by this thread (empty if none). */
const char* ss_last_error_string(void);
const char* ss_version(void);

/* ------------------------------------------------------- maximum mipmap
 * Sec. 3.2 "Maximum mipmaps": level 0 is the heightfield; level l+1 has
 * ceil(w/2) x ceil(h/2) texels, each the maximum of the (up to) 2x2 texels of
 * level l below it; levels continue down to 1x1.  The library stores levels
 * 1..L-1 in one caller-allocated device buffer: level l starts at element
 * offset_elems (256-byte aligned) and has row stride pitch (a multiple of 4
 * elements).  Three 32-bit words follow the levels: [stats] = (global max,
 * global min) of the heightfield as float32 (NaN texels ignored), and the
 * number of non-finite texels as a uint32. */
int32_t ss_maxmip_levels(int32_t nx, int32_t ny);          /* L, or 0 on bad size */
size_t ss_maxmip_bytes(int32_t nx, int32_t ny);            /* 0 on bad size       */
ss_status ss_maxmip_level_info(int32_t nx, int32_t ny, int32_t level, int32_t* width,
                               int32_t* height, int64_t* pitch, int64_t* offset_elems);
/* Builds every level of hf->h's pyramid into mip (device, ss_maxmip_bytes).
 * Bit-exact: each texel is exactly one of the input values. */
ss_status ss_build_maxmip(const ss_heightfield* hf, float* mip, ss_stream_t stream);

/* ----------------------------------------------------------- forward
 * Exact descent over the maximum mipmap (Sec. 3.2 "Dynamic Programming",
 * Eq. optimumk2: the clearance over an interval is bounded through the maximum
 * height below it).  Aligned blocks of samples are bounded by the mip maximum
 * over their texel footprint; blocks whose bound cannot beat the running
 * minimum are skipped; the rest are split until single samples are evaluated.
 * Sample values are float32 in a per-ray local frame (FP64 per-ray setup); the
 * argmin sample of rays with unsaturated light is re-evaluated in FP64.
 * mip: device, built by ss_build_maxmip for the same heights. */
ss_status ss_shadow_forward(const ss_heightfield* hf, const float* mip, const ss_rays* rays,
                            const ss_sun* sun, const ss_params* params,
                            const ss_outputs* out, ss_stream_t stream);

/* Uniform ray stepping (Sec. 2, Fig. 1b): every usable sample in order, with an
 * exact early exit once (H(t) - max h)/t, non-decreasing in t, reaches the
 * running minimum.  Same sample values as ss_shadow_forward, so both return the
 * same argmin and cost bit for bit.  mip: used only for the global max. */
ss_status ss_shadow_uniform(const ss_heightfield* hf, const float* mip, const ss_rays* rays,
                            const ss_sun* sun, const ss_params* params,
                            const ss_outputs* out, ss_stream_t stream);

/* ---------------------------------------------------------- backward
 * Adjoint of light with respect to the heights and the sun direction, at each
 * ray's forward argmin (a subgradient of the minimum; derived from Eq. discfrac
 * and the sample cost).  Inputs: argmin from ss_shadow_forward; cost (optional,
 * device [n] float32, the forward's cost output) lets rays whose light is
 * certainly saturated (zero gradient) be skipped before any FP64 work;
 * grad_light (device [n] float32, dLoss/dlight).  grad_h (device, [ny][pitch]
 * float32) is ACCUMULATED into (zero it first); grad_sun (device double[5]) is
 * accumulated: (dL/d elevation, dL/d azimuth, dL/ds_x, dL/ds_y, dL/ds_z), s a
 * free 3-vector.  Rays with j* = -1 or saturated light contribute nothing.
 * Atomic accumulation: summation order, and so the last bits, may vary
 * between runs (float32 atomics on grad_h, FP64 on grad_sun).
 * params->flags must not hold SS_FLAG_DETERMINISTIC_BWD (use
 * ss_shadow_backward_ws). */
ss_status ss_shadow_backward(const ss_heightfield* hf, const ss_rays* rays, const ss_sun* sun,
                             const ss_params* params, const int32_t* argmin, const float* cost,
                             const float* grad_light, float* grad_h, double* grad_sun,
                             ss_stream_t stream);

/* ss_shadow_backward with a caller workspace, a status word and, with
 * SS_FLAG_DETERMINISTIC_BWD in params->flags, results that are the same bits
 * on every run and every launch shape (no counterpart in the paper; it makes
 * a training loop over heights reproducible).  Deterministic mode, two passes
 * over the rays that need FP64 work:
 *   1. each contribution to a texel counts into that texel (integer atomics)
 *      and the largest |contribution| and the largest count are kept;
 *   2. a power-of-two scale 2^S with (largest |contribution|) (largest count)
 *      2^S < 2^62 is chosen, every contribution is rounded to the integer
 *      nearest its value times 2^S and summed in 64-bit integers (exact, so the
 *      order cannot matter), and grad_h += (float)(sum 2^-S) per texel.
 *   The sun gradient is summed the same way (scale from the largest |value|
 *   and the number of rays) and added to grad_sun.
 *   Error: each texel's sum is exact up to (count) 2^-(S+1) from the
 *   rounding to integers, far below the float32 rounding of the result.
 * Without the flag the call behaves as ss_shadow_backward (workspace unused).
 * workspace: device, at least ss_backward_workspace_bytes(nx, ny, flags)
 * bytes, 256-byte aligned, not in use by another call in flight.
 * status: optional device word OR-ed with SS_DEV_NONFINITE_GRAD when a
 * dL/dlight value is non-finite (that ray is skipped), or NULL.
 * Errors: as ss_shadow_backward; short or NULL workspace in deterministic
 * mode -> SS_ERR_OUT_OF_MEMORY / SS_ERR_INVALID_ARG. */
size_t ss_backward_workspace_bytes(int32_t nx, int32_t ny, uint32_t flags);
ss_status ss_shadow_backward_ws(const ss_heightfield* hf, const ss_rays* rays, const ss_sun* sun,
                                const ss_params* params, const int32_t* argmin,
                                const float* cost, const float* grad_light, float* grad_h,
                                double* grad_sun, void* workspace, size_t workspace_bytes,
                                uint32_t* status, ss_stream_t stream);

/* ------------------------------------------------------------- batched
 * Many (heightfield tile, sun) instances of uneven sizes in one persistent
 * launch: the maximum mipmaps of all instances are built, then one kernel with
 * a device-side work queue (a chunk counter in the workspace; no device-side
 * waits) walks every ray of every instance with the exact descent of
 * ss_shadow_forward, giving the same per-ray outputs bit for bit.  The nearest
 * counterpart in the paper is drawing many visible tiles per frame (Sec. 3.3,
 * virtual texturing; Sec. 6.3).  Grid-mode rays (one per texel centre),
 * gnomonic tiles.  params (max_len_m, step_texels, ...) apply to every item;
 * zero shape fields take the batch defaults: exact walks in 64 x 64 chunks of
 * texels (rays_per_thread 128, ray_tile_w 64) with column seeds and services
 * at 14 idle lanes, light-only walks in runs of 512 (rays_per_thread 16) with
 * services at 6.  A caller who sets rays_per_thread sets ray_tile_w too
 * (0 = runs of consecutive texels). */
typedef struct {
    ss_heightfield hf;     /* device heights; projection SS_PROJ_GNOMONIC       */
    float* mip;            /* device, ss_maxmip_bytes(hf.nx, hf.ny); written    */
    ss_sun sun;
    ss_outputs out;        /* device arrays of hf.nx * hf.ny entries            */
} ss_batch_item;

/* Bytes of the device workspace a batch of n_items needs (caller-allocated;
 * holds the instance descriptors and the work-queue counter). */
size_t ss_batch_workspace_bytes(int32_t n_items);

/* Enqueue one batch on `stream`: descriptor upload (from host memory, copied
 * before the call returns), queue reset, mipmap builds, persistent kernel.
 * The workspace must not be in use by another batch in flight. */
ss_status ss_batch_submit(const ss_batch_item* items, int32_t n_items, const ss_params* params,
                          void* workspace, size_t workspace_bytes, ss_stream_t stream);

/* A batch captured once into a CUDA graph and replayed: plan_create uploads the
 * descriptors (synchronously) and captures queue reset + mipmap builds +
 * persistent kernel; plan_launch replays the graph on `stream` (the items'
 * buffers and the workspace must stay valid while the plan exists, and
 * replays of one plan must not overlap). */
typedef struct ss_batch_plan ss_batch_plan;
ss_status ss_batch_plan_create(const ss_batch_item* items, int32_t n_items,
                               const ss_params* params, void* workspace, size_t workspace_bytes,
                               ss_batch_plan** plan);
ss_status ss_batch_plan_launch(ss_batch_plan* plan, ss_stream_t stream);
ss_status ss_batch_plan_destroy(ss_batch_plan* plan);

/* ss_batch_submit without any device allocation (no counterpart in the paper;
 * an interface for callers that cannot allocate).  Some callers cannot give the
 * batch a workspace: a renderer's frame loop that must not call cudaMalloc
 * (it may synchronise the device and stall the frame), or a host program
 * whose device memory belongs to another allocator.  This entry point keeps
 * the workspace in a fixed array of ss_batch_static_scratch_bytes() bytes in
 * the library's device image instead (every GPU that loads the library holds
 * it until the process exits) and otherwise behaves as ss_batch_submit.
 * Limit: at most SS_BATCH_STATIC_MAX_ITEMS items; more returns SS_ERR_BAD_SIZE
 * (message in ss_last_error_string()).  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) for that device; make
 * that first call before any stream capture.  Every call reuses the same
 * array, overwriting the previous call's descriptors and resetting its queue
 * counter: calls that overlap on the GPU (different streams, not ordered)
 * race and give wrong results; order them on one stream or synchronise.
 * Calls no cudaMalloc/cudaFree or other allocating routine. */
#define SS_BATCH_STATIC_MAX_ITEMS 256
size_t ss_batch_static_scratch_bytes(void);
ss_status ss_batch_submit_static(const ss_batch_item* items, int32_t n_items,
                                 const ss_params* params, ss_stream_t stream);

/* ------------------------------------------------------ greedy descent --
 * The paper's own greedy descent (Algorithm 1, ray length T of Eq. maxstep,
 * interval concatenation of Sec. 3.3 "Long shadows"), an APPROXIMATION of the
 * minimum that ss_shadow_forward computes exactly; provided to reproduce the
 * paper's method and measure its error.  Run r covers [a_r, a_r + T_r] with
 * N'_r = levels[r] mip levels: T_r is the ray parameter closest to the line
 * from the sphere's centre through the texel point 2^(N'_r - 1) texels from the
 * run start's texel image along the unit texture-plane direction of (s_x, s_y);
 * with t in [0, 1] over the run, level k = 0 .. N'_r - 1 reads maximum-mipmap
 * level N'_r - 1 - k (the texel containing the tip's texel image, no filtering)
 * at t_k, t_k - 2^-(k+1), t_k - 2^-k (t_0 = 1), keeps the smallest
 * Delta = tip height over the sphere - M (first on ties; tips at t <= 0 or off
 * the tile are skipped) and continues from t* + 2^-(k+1); the run's cost is the
 * last level's Delta* over its distance, the ray's the smallest run cost.
 * light as for ss_shadow_forward.  All in FP64.
 * Inputs: hf, mip (ss_build_maxmip), rays (grid or list), sun; levels[n_runs]
 * (host), 1 <= n_runs <= SS_GREEDY_MAX_RUNS, 1 <= levels[r] <=
 * ss_maxmip_levels(nx, ny).  Outputs (device, one per ray): light; cost (rad,
 * +inf when no tip was read) and t_star (m, -1 then) optional (NULL).
 * Errors: as ss_shadow_forward for hf, rays and sun; bad levels/n_runs ->
 * SS_ERR_INVALID_ARG. */
#define SS_GREEDY_MAX_RUNS 8
ss_status ss_shadow_greedy(const ss_heightfield* hf, const float* mip, const ss_rays* rays,
                           const ss_sun* sun, const int32_t* levels, int32_t n_runs,
                           float* light, float* cost, float* t_star, ss_stream_t stream);

/* The same greedy descent at the arithmetic of the paper's shader (float32,
 * Sec. 6.3), gnomonic tiles only (SS_ERR_UNSUPPORTED otherwise): tip heights in
 * the ray's local frame, tip texel images from the ray's float32 slope, the run
 * length of Eq. maxstep in float32; FP64 only where a tip's float32 image lies
 * within its error margin of a mip-cell edge or of the tile's border.  Its
 * decisions can differ from ss_shadow_greedy's where tips nearly tie; arguments
 * and outputs as ss_shadow_greedy. */
ss_status ss_shadow_greedy_f32(const ss_heightfield* hf, const float* mip, const ss_rays* rays,
                               const ss_sun* sun, const int32_t* levels, int32_t n_runs,
                               float* light, float* cost, float* t_star, ss_stream_t stream);

/* ----------------------------------------------------- shading epilogue --
 * Lambertian irradiance of the terrain under several disc lights (Sec. 3.4:
 * the Sun and the Earth are discs and each has its own lit fraction s_l, from
 * ss_shadow_forward with that light as the "sun"; Sec. 6.3: Lambertian BRDF):
 *   E = sum_l intensity_l * s_l * max(0, N . L_l)
 * L_l from elevation/azimuth as for ss_sun; N the unit normal of the terrain
 * surface r(u, v) = (R + h(u, v)) n(u, v) at the ray origin: grid rays take
 * h_u, h_v as central differences of the texel values (one-sided on the
 * border), listed rays the gradient of the bilinear interpolant in their cell
 * (lift is ignored: the normal is the terrain's).  float32.
 * Inputs: hf, rays (as for ss_shadow_forward); lights[n_lights] (host array,
 * 1 <= n_lights <= SS_SHADE_MAX_LIGHTS) whose `lit` arrays are device float
 * [n rays].  Output: irradiance (device float [n rays]).
 * Errors: as ss_shadow_forward for hf and rays; bad lights -> SS_ERR_INVALID_ARG. */
#define SS_SHADE_MAX_LIGHTS 8
typedef struct {
    double elevation_rad, azimuth_rad;   /* light direction (tile-centre frame)     */
    double intensity;                    /* irradiance at normal incidence, unlit 0 */
    const float* lit;                    /* device: lit fraction per ray            */
} ss_light;

ss_status ss_shade(const ss_heightfield* hf, const ss_rays* rays, const ss_light* lights,
                   int32_t n_lights, float* irradiance, ss_stream_t stream);

/* ------------------------------------------------------------ view rays --
 * The terrain points a camera sees: the origins of the shadow rays of a view
 * (Sec. 4: view rays are intersected with the displaced terrain; the maximum
 * mipmap lets a ray skip the sample blocks it passes above).
 *
 * Pixel (i, j), row 0 at the top, W = width, H = height, looks along
 *   d = unit(forward + a right + b up), a = (2(i + 0.5)/W - 1) tan_half_x,
 *   b = (1 - 2(j + 0.5)/H) tan_half_y.
 * Along x(tau) = pos + tau d the samples tau_k = k step_m, k = 1 ..
 * floor(max_dist_m / step_m), are tested in order; the hit is the first one
 * whose texel image lies in [0,nx-1] x [0,ny-1] with |x| - R - h(image) <= 0
 * (h bilinear, decided in FP64); when the sample before it is in the tile too
 * the crossing is refined in FP64: bisection of that step until the bracket
 * lies in one bilinear cell, then the single root there of the quadratic that
 * |x| - R - h is along the ray within one cell, placed within 8x the FP64
 * rounding of that difference over its slope (within a third of a float32
 * step of the texel coordinates; points within 0.25 texel of the tile's low
 * edges, and near-tangent crossings, bisect on to 2^-36 of the step).  The
 * march itself runs in float32 and defers to FP64 near the terrain and the
 * tile's border.
 *
 * Output: the hits' texel coordinates (u, v) as float32 pairs in pixel order,
 * uv[2*r], uv[2*r+1] for r < *count (device int64 written by the call), and
 * optionally pixel[r] = j*W + i.  Pixels without a hit (sky, off the tile)
 * produce no entry.  The list feeds ss_shadow_forward as SS_RAYS_LIST rays
 * (lift 0).  Sizes: uv holds 2*W*H floats, pixel W*H ints; workspace
 * ss_view_workspace_bytes(W, H) bytes (caller-allocated, device).
 * Errors: W, H < 1 or W*H >= 2^31 -> SS_ERR_BAD_SIZE; non-finite camera
 * numbers, step_m <= 0, max_dist_m <= 0, more than 2^31 samples, NULL
 * pointers or a short workspace -> SS_ERR_INVALID_ARG / SS_ERR_BAD_SIZE. */
typedef struct {
    double pos[3];                      /* camera centre, tile frame (m)          */
    double forward[3], right[3], up[3]; /* orthonormal view frame                 */
    double tan_half_x, tan_half_y;      /* tangents of the half fields of view   */
    int32_t width, height;              /* pixels                                 */
} ss_camera;

size_t ss_view_workspace_bytes(int32_t width, int32_t height);
ss_status ss_view_rays(const ss_heightfield* hf, const float* mip, const ss_camera* cam,
                       double step_m, double max_dist_m, float* uv, int32_t* pixel,
                       int64_t* count, void* workspace, size_t workspace_bytes,
                       ss_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* SOFTSHADOW_H */
