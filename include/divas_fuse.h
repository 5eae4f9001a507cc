/*
 * divas_fuse.h -- C ABI of the depth-weighted multi-view voxel fusion
 * (DivAS, arXiv 2601.04860) on NVIDIA B300 (sm_103a).
 *
 * The operation (Sec. 3.5 "Shared voxel-voting concept"; Eq. compact-fusion,
 * Eq. gs-depthweight, Eq. vmask; the thick-path algorithms of Appendix A.2
 * "Thick-Structure Segmentation via Depth-Weighted Voxel Aggregation" and
 * Appendix B.5 "Thick-Structure Segmentation for 2DGS"): for every voxel v
 * of an occupied set (centre x_v, edge h_v) and every view i in order,
 *
 *   p = R_i x_v + t_i;  skip unless p_z > z_near
 *   u = fx p_x/p_z + cx, v = fy p_y/p_z + cy; skip unless 0 <= u < W, 0 <= v < H
 *   D = depth_i[floor v][floor u], m = mask_i[floor v][floor u]
 *   skip unless D is finite and > 0, and m >= tau_mask
 *   Delta = gamma h_v, e = p_z - D; skip unless |e| <= Delta
 *   w = exp(-alpha1 (e/Delta)^2);  W += m w;  Z += w;  bits |= 1 << i
 *
 * then P = W/Z (Z > eps, else 0), seg = P >= tau_cons, vmask = seg ? bits : 0,
 * and points are labelled by the seg bit of the voxel containing them
 * (Eq. pass1).  Arithmetic is FP32 with a compensated depth residual; see
 * the package documentation for the error analysis.
 *
 * Conventions
 *   - Grid: voxel (i, j, k) centre = origin + (idx + 1/2) h; linear index
 *     (k g + j) g + i (x fastest).  A contracted grid covers contracted space
 *     [-2, 2]^3 (unbounded scenes): centres are uncontracted with
 *     x = c / (|c| (2 - |c|)) for 1 < |c| < 2 (x = c inside the unit ball),
 *     h_v = h / (2 - |c|)^2 there; voxels with |c| >= 2 never vote.  Points
 *     are contracted with (2 - 1/|x|) x/|x| before lookup.
 *   - Camera: OpenCV world->camera (x right, y down, z forward), R row-major;
 *     pixel (i, j) covers [i, i+1) x [j, j+1); rasters are row-major H x W.
 *   - Depth: planar camera-Z, float32; +inf, NaN or <= 0 means no surface.
 *   - Views of one context are numbered 0, 1, 2, ... in the order they are
 *     added; bit i of vmask is view i (views from 32 on vote but set no bit).
 *
 * Ownership and streams
 *   Every pointer argument marked "device" is a CUDA device pointer owned by
 *   the caller, which must keep it valid until the work queued on `stream`
 *   has consumed it (the usual CUDA asynchronous contract).  Host structs
 *   are copied during the call.  `stream` is a cudaStream_t (NULL = legacy
 *   default stream).  The context owns its device state (accumulators,
 *   active list, occupancy rank structure, seg bitfield).  Calls on one
 *   context must not run concurrently from several host threads.
 *
 * Errors
 *   Every call returns a divas_status and never aborts.  Invalid arguments
 *   return DIVAS_E_INVALID before any work is queued; CUDA launch or
 *   allocation failures return DIVAS_E_CUDA / DIVAS_E_OOM.  Conditions found
 *   on the device (a sparse coordinate outside the grid, an occupied set
 *   larger than the context's capacity) are recorded in a device status
 *   word and returned by the next call that synchronises (divas_fuse_finalize
 *   with a non-NULL n_seg_host, or divas_fuse_sync).  divas_last_error gives
 *   a message for the last failing call on the context.
 */
#ifndef DIVAS_FUSE_H
#define DIVAS_FUSE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct divas_ctx divas_ctx;

typedef enum {
    DIVAS_OK = 0,
    DIVAS_E_INVALID = 1,  /* bad argument; nothing was queued */
    DIVAS_E_OOM = 2,      /* device allocation failed */
    DIVAS_E_CUDA = 3,     /* a CUDA call failed (message in divas_last_error) */
    DIVAS_E_TIMEOUT = 4,  /* reserved: no kernel of this library waits on another CTA */
    DIVAS_E_STATE = 5,    /* call not valid in the context's current state */
    DIVAS_E_CAPACITY = 6  /* occupied set larger than the context's capacity */
} divas_status;

typedef enum {
    DIVAS_MASK_F32 = 0,      /* float32 probability in [0, 1] */
    DIVAS_MASK_F16 = 1,      /* IEEE binary16 probability (widened exactly) */
    DIVAS_MASK_LOGIT_F32 = 2 /* float32 logit l; m = 1/(1+exp(-l)); gate l >= logit(tau_mask) */
} divas_mask_t;

/* Constants of the thick path.  Defaults (divas_default_params): tau_mask 0.5
 * (thick-path entry m >= 0.5, Algorithms A.2/B.5), gamma 1.0 and tau_cons 0.5
 * (Table gs-hyperparams), alpha1 0.5 and eps 1e-12 (the paper gives no
 * values), z_near 1e-6. */
typedef struct {
    float tau_mask, gamma, alpha1, tau_cons, eps, z_near;
    uint32_t flags; /* 0 or DIVAS_ORDER_BRICKS */
} divas_params;

/* divas_params.flags: the active list in brick-major order instead of
 * ascending linear index -- 8 x 8 x 8 bricks in linear brick order (x
 * fastest), the cells of a brick in linear order (x fastest).  Either prior
 * kind (a dense prior 8-byte aligned), g a multiple of 8 (else
 * DIVAS_E_INVALID).  Every per-voxel result is
 * unchanged; only the order of the active list, and so of everything stored
 * or returned in active-list order, differs.  Consecutive active voxels then
 * lie close together in space, which lets the fusion skip, for a whole warp of
 * voxels, a view whose mask gate none of them can pass (see
 * divas_fuse_add_views). */
#define DIVAS_ORDER_BRICKS 1u


typedef struct {
    int32_t kind;       /* 0: dense prior (occ_dense), 1: sparse prior (coords) */
    int32_t g;          /* voxels per side, 1 <= g <= 1024 */
    float origin[3], h; /* voxel (i,j,k) centre = origin + (idx + 1/2) h, h > 0 */
    int32_t contracted; /* 1: the grid lives in contracted space (see above) */
} divas_grid;

typedef struct {
    int32_t W, H;       /* raster size, 1..65535 each */
    float fx, fy, cx, cy;
    float R[9], t[3];   /* world -> camera, row-major */
} divas_camera;

typedef struct {
    divas_camera cam;
    const float* depth; /* device, H x W float32 planar depth */
    const void* mask;   /* device, H x W, element type from mask_type */
    int32_t mask_type;  /* divas_mask_t */
    int32_t reserved;
} divas_view;

/* Largest number of views one divas_fuse_add_views call accepts. */
#define DIVAS_MAX_VIEWS_PER_CALL 32

void divas_default_params(divas_params* out);

/*
 * Create a context for one occupied set and build its active list (the
 * occupancy-prior gate and active-voxel list of Sec. 3.5 "Occupancy by
 * Morton-scattered opacity" and Appendix B.1).
 *   kind 0: occ_dense = device g^3 uint8 (x fastest), nonzero = occupied;
 *           coords must be NULL.
 *   kind 1: coords = device n_coords x 3 int32 (i, j, k); duplicates are
 *           merged; occ_dense must be NULL.
 * The active list is ordered by ascending linear index (brick-major with
 * DIVAS_ORDER_BRICKS).  Allocates device
 * memory and synchronises `stream` once (to size the active arrays).
 */
divas_status divas_fuse_init(divas_ctx** out, const divas_grid* grid, const uint8_t* occ_dense,
                             const int32_t* coords, int64_t n_coords, const divas_params* params,
                             void* stream);

/* Rebuild the active list from a new prior of the same kind and grid, reusing
 * the context's memory (no allocation, no synchronisation); the view count
 * returns to 0, so the next fold starts the accumulators from zero, and the
 * context's seg bitfield is cleared (labels read 0 until the next finalize).
 * If the new occupied set exceeds the capacity sized at init, the excess
 * voxels are dropped and DIVAS_E_CAPACITY is reported by the next
 * synchronising call. */
divas_status divas_fuse_set_occupancy(divas_ctx* ctx, const uint8_t* occ_dense,
                                      const int32_t* coords, int64_t n_coords, void* stream);

/* Fold one view into the accumulators (incremental update). */
divas_status divas_fuse_add_view(divas_ctx* ctx, const divas_camera* cam, const float* depth,
                                 const void* mask, int32_t mask_type, void* stream);

/* Fold n_views (1..DIVAS_MAX_VIEWS_PER_CALL) views in index order in one
 * launch.  The result is bitwise identical to n_views add_view calls. */
divas_status divas_fuse_add_views(divas_ctx* ctx, const divas_view* views, int32_t n_views,
                                  void* stream);

/*
 * Normalise and threshold (Eq. compact-fusion, V_seg = {P >= tau_cons}).
 *   score_out    device float32: dense kind -> g^3 (0 for unoccupied voxels);
 *                sparse kind -> n_active, in active-list order.  Nullable.
 *   seg_bits_out device uint32, ceil(g^3 / 32) words, bit (lin & 31) of word
 *                (lin >> 5) = seg of voxel lin (0 for unoccupied).  Nullable.
 *   vmask_out    device uint32, n_active, in active-list order.  Nullable.
 *   n_seg_host   host int64: number of segmented voxels.  Nullable; non-NULL
 *                synchronises the stream and reports device-side errors.
 * The context keeps its own seg bitfield for divas_label_points.
 */
divas_status divas_fuse_finalize(divas_ctx* ctx, float* score_out, uint32_t* seg_bits_out,
                                 uint32_t* vmask_out, int64_t* n_seg_host, void* stream);

/* flags of divas_fuse_update and divas_batch_finalize */
#define DIVAS_KEEP_ZEROS 1u /* score_out / seg_bits_out already hold 0 for every unoccupied
                               voxel (e.g. an earlier result of this context for the same
                               occupied set): only the active voxels' entries are written */

/*
 * Incremental update (Sec. 3.7: a new view arrives and the 3D mask is shown
 * again): fold n_views (1..DIVAS_MAX_VIEWS_PER_CALL) views onto the stored
 * accumulators and finalize, in one fusion launch.  Results equal
 * divas_fuse_add_views followed by divas_fuse_finalize (score_out and
 * seg_bits_out as there, nullable; no vmask, no count).  Without
 * DIVAS_KEEP_ZEROS a dense score_out also gets its unoccupied zeros (in the
 * same launch) and seg_bits_out is cleared first; with it, only active
 * entries are written and bits are set and cleared in place.
 */
divas_status divas_fuse_update(divas_ctx* ctx, const divas_view* views, int32_t n_views,
                               float* score_out, uint32_t* seg_bits_out, uint32_t flags,
                               void* stream);

/*
 * The whole hot path in one call: divas_fuse_set_occupancy (A1), then
 * divas_fuse_add_views (views folded into fresh accumulators), then finalize
 * (score_out, seg_bits_out as in divas_fuse_finalize) and, when n_pts > 0,
 * divas_label_points, in four launches for a dense prior in linear order (a
 * sparse prior adds the bitfield's memset and the coordinate scatter, view
 * culling two more) and no memset of the outputs: the compaction clears
 * the seg bitfields, and the fusion launch also normalises and thresholds
 * each voxel and then writes the zeros of a dense score_out's unoccupied
 * cells.  Results (outputs and
 * context state) equal the separate calls; 1..DIVAS_MAX_VIEWS_PER_CALL views.
 * Capturable in a CUDA graph.  A brick-ordered context fusing at least four
 * views also launches its two culling kernels (mask pyramids, brick test) on
 * a helper stream of its own, forked from `stream` at the call's start and
 * joined back before the fusion by events (a captured step holds them as a
 * parallel branch); the call's work is ordered after earlier work on
 * `stream` and before later work on it, as for a single-stream call.  If the
 * occupied set overflows the capacity
 * (DIVAS_E_CAPACITY at the next synchronising call), the dense scores of the
 * dropped voxels are unspecified.
 */
divas_status divas_fuse_step(divas_ctx* ctx, const uint8_t* occ_dense, const int32_t* coords,
                             int64_t n_coords, const divas_view* views, int32_t n_views,
                             float* score_out, uint32_t* seg_bits_out, const float* xyz,
                             int64_t n_pts, uint8_t* labels_out, void* stream);

/* divas_fuse_step that also records stage_events[k] (cudaEvent_t, entries
 * nullable; the array nullable) on `stream`: [0] before the compaction, [1]
 * after it, [2] after the fusion + finalize launch, [3] after the labels.
 * During a stream capture they become external event-record nodes (events
 * created with timing enabled time a graph replay's stages). */
divas_status divas_fuse_step_profiled(divas_ctx* ctx, const uint8_t* occ_dense,
                                      const int32_t* coords, int64_t n_coords,
                                      const divas_view* views, int32_t n_views, float* score_out,
                                      uint32_t* seg_bits_out, const float* xyz, int64_t n_pts,
                                      uint8_t* labels_out, void* const* stage_events,
                                      void* stream);

/*
 * Depth-tuple mode (Sec. 3.5 "Planar-to-ray depth correction" .. "Thin-
 * structure path"; Algorithms "Thick-Structure Segmentation for 2DGS" and
 * "Thin-Structure Segmentation for 2DGS", Appendix B.5).  Each view carries
 * the renderer's depth tuple instead of one depth: the thick path takes the
 * footprint statistics of n_samp (integral images), the layered / see-through
 * / trust tests, the asymmetric depth gate with the count-tightened tolerance
 * gamma h_v / (1 + beta E), the ray-space spatial gate with the depth-gradient
 * factor and the depth-band weight; a view that casts no thick vote and passes
 * the behind-surface gate goes through the thin path over the voxel's
 * projected footprint (two counters, coverage, peak mask, distance gate) and
 * adds its score t to W and 1 to Z when t >= tau_thin.  The occupied set is
 * binary (density 1 per active voxel).
 */
typedef struct {
    divas_camera cam;
    const float* d_min;      /* device H x W planar depths (front hit, median, back); */
    const float* d_med;      /* +inf, NaN or <= 0: no surface                           */
    const float* d_max;
    const uint16_t* n_samp;  /* device H x W splat-traversal count                       */
    const void* mask;        /* device H x W, as in divas_view                           */
    int32_t mask_type;
    float d_cam;             /* camera-target distance (see-through test)                */
} divas_tuple_view;

typedef struct {
    float beta;          /* count tightening (0.05)                                       */
    float gamma_st;      /* see-through threshold as a multiple of d_cam (1.5)             */
    float tau_thin;      /* thin-path acceptance (0.6); must be > 0                       */
    float rho_cover;     /* coverage n_md / n_depth (0.5)                                 */
    float rho_occ;       /* fractional support floor of the footprint area (0.1)           */
    float n_abs;         /* absolute support floor (25)                                   */
    float dist_gate;     /* unprojection distance gate in units of h_v (1.5)               */
    float behind_margin; /* behind-surface margin in units of h_v (2)                      */
    float k_dg;          /* depth-gradient decay (0: factor 1)                             */
    float rho_thin;      /* thin-path density floor (1: every active voxel is eligible)    */
} divas_tuple_params;

/* The constants above (Table gs-hyperparams; k_dg and rho_thin are readings). */
divas_tuple_params divas_default_tuple_params(void);

/* Fold n_views (1..DIVAS_MAX_VIEWS_PER_CALL) tuple views in index order onto
 * the accumulators (view bits continue the context's count); finalize as
 * usual.  Footprint sums of n_samp come straight from the raster when the
 * grid's geometry bounds every footprint of a view to at most 256 pixels,
 * else from per-view integral images built in context scratch that grows on
 * demand (the first call that needs more allocates and synchronises; such a
 * call inside a stream capture returns DIVAS_E_STATE).  Integral-image sums
 * are exact for footprints below 2^16 pixels.  DIVAS_E_INVALID: NULL or
 * out-of-range arguments (including tau_thin <= 0, where a view without thin
 * evidence would add a zero vote), before any launch. */
divas_status divas_fuse_add_views_tuple(divas_ctx* ctx, const divas_tuple_view* views,
                                        int32_t n_views, const divas_tuple_params* tp,
                                        void* stream);

/* divas_fuse_add_views_tuple that also records stage_events[k] (cudaEvent_t,
 * entries nullable; the array nullable) on `stream`: [0] before the per-view
 * maps (mask-tile maxima, integral images), [1] after them, [2] after the
 * candidate scan of the last 16-view batch, [3] after its heavy pass.  Inside
 * a stream capture they become external event-record nodes. */
divas_status divas_fuse_add_views_tuple_profiled(divas_ctx* ctx, const divas_tuple_view* views,
                                                 int32_t n_views, const divas_tuple_params* tp,
                                                 void* const* stage_events, void* stream);

/*
 * NeRF variant of the depth-tuple fusion (appendix "NeRF-Backbone 3D Fusion
 * Details": Eqs. distance_cond, dist_tol, depth_tol, nerf-accept, nerf-vote,
 * nerf-thindepth .. nerf-thin; Algorithms "Thick-Structure Segmentation via
 * Depth-Weighted Voxel Aggregation" and "Thin-Structure Segmentation via
 * Footprint-Based Coverage Analysis").  Views are divas_tuple_view with
 * d_med holding the expected depth d_exp (d_min, d_exp, d_max planar; n_samp
 * the ray-sample count; d_cam unused).  Per voxel (edge Delta) and view:
 *   thick, at the centre pixel (x, y) when m >= tau_m and the three depths
 *   are finite and positive: k = ((x + 1/2 - cx)/fx, (y + 1/2 - cy)/fy, 1)
 *   (the pixel-centre ray; a planar depth d on it is the point k d), p the
 *   camera-space voxel centre, z_c = clip(<p, k> / |k|^2, d_min, d_max)
 *   (clip(z, a, b) = a if z < a, else b if z > b, else z; also for b < a),
 *   delta = |p - k z_c| <= Delta pi_dg + lambda_range |k| (d_max - d_min) and
 *   |p_z - d_exp| <= (gamma + min(beta n, b_max)) Delta: W += m w, Z += w,
 *   w = exp(-alpha1 r^2), r = |z_c - (d_min + d_max)/2| / max((d_max -
 *   d_min)/2, eps);
 *   thin, when the thick path did not vote, m > m_thin (logits: l >
 *   logit(m_thin) in FP32) and the voxel's density >= rho_thin: over the box
 *   of the 8 projected corners clipped to the frame (N pixels), n_valid = #
 *   {q: m(q) > 1/2 and |p_z - d_exp(q)| <= (2 gamma + min(beta n(q), b_max))
 *   Delta}, m_max = max m(q); t = m_max if n_valid >= rho_cover N, else 0;
 *   t >= tau_thin: W += t, Z += 1.
 * gamma here replaces the context's gamma; alpha1, tau_m, eps and z_near
 * are the context's.
 */
enum { DIVAS_NERF_LLFF = 0, DIVAS_NERF_MIP360 = 1 };

typedef struct {
    float gamma;         /* base tolerance multiplier (4.0 LLFF, 0.5 Mip-NeRF 360)          */
    float beta;          /* per-sample bonus (0.2)                                         */
    float b_max;         /* bonus cap (10, 1)                                              */
    float lambda_range;  /* band slack of the spatial tolerance (0.05, 5.0)                */
    float rho_thin;      /* thin-path density floor (50, 30)                               */
    float rho_cover;     /* thin coverage threshold (0.20, 0.30)                           */
    float tau_thin;      /* thin acceptance (0.6); must be > 0                             */
    float m_thin;        /* thin eligibility of the centre mask (0.1), in [0, 1)           */
    float k_dg;          /* depth-gradient decay (0: factor 1)                             */
    int32_t reserved;
} divas_nerf_params;

/* Table kernel_hyperparams' column for DIVAS_NERF_LLFF or DIVAS_NERF_MIP360
 * (any other value: LLFF); m_thin from the thin path's eligibility rule,
 * k_dg = 0 a reading (no value given). */
divas_nerf_params divas_default_nerf_params(int32_t preset);

/* Fold n_views (1..32) NeRF tuple views in index order onto the
 * accumulators; finalize as usual.  density: NULL (every active voxel has
 * density 1) or device g^3 FP32 (x fastest, 4-byte aligned), read for the
 * thin path's floor.  Scratch (the heavy list, mask-tile maxima) is the
 * tuple mode's, grown on demand (outside a stream capture, else
 * DIVAS_E_STATE).  DIVAS_E_INVALID: NULL or out-of-range arguments, before
 * any launch. */
divas_status divas_fuse_add_views_nerf(divas_ctx* ctx, const divas_tuple_view* views,
                                       int32_t n_views, const divas_nerf_params* np,
                                       const float* density, void* stream);

/* The same, recording stage_events[k] (cudaEvent_t, nullable) on stream: [0]
 * before the mask-tile maps, [1] after them, [2] after the scan of the last
 * 16-view batch, [3] after its heavy pass. */
divas_status divas_fuse_add_views_nerf_profiled(divas_ctx* ctx, const divas_tuple_view* views,
                                                int32_t n_views, const divas_nerf_params* np,
                                                const float* density, void* const* stage_events,
                                                void* stream);

/* The density floor of the NeRF occupancy (the empty-voxel skip of
 * Algorithm "Thick-Structure Segmentation via Depth-Weighted Voxel
 * Aggregation"): occ[i] = density[i] >= rho_thresh (1 / 0; NaN gives 0),
 * the uint8 prior divas_fuse_set_occupancy takes.  density: device n FP32,
 * 16-byte aligned; occ: device n uint8, 4-byte aligned; DIVAS_E_INVALID
 * otherwise.  Asynchronous on stream. */
divas_status divas_density_floor(const float* density, int64_t n, float rho_thresh, uint8_t* occ,
                                 void* stream);

/*
 * Depth-weighted mask refinement (Sec. 3.4 "Depth-weighting: bounded
 * normalization (NeRF) vs. band-pass (2DGS)"), a per-view pre-pass whose
 * output is folded like any FP32 mask (add_views, add_views_tuple, update):
 *   DIVAS_WEIGHT_NERF_MINMAX (Eq. nerf-depthweight): M~ = M (1 - Z^),
 *     Z^ = (D - min D) / (max D - min D) over the view's depth raster D;
 *   DIVAS_WEIGHT_GS_BAND (Eqs. depthband, gs-bandpass): [d_min, d_max] = the
 *     range of D at the positive prompts and at the view centre pixel
 *     (W / 2, H / 2) (integer halves), d_far = P98(D) (linear interpolation
 *     between the order statistics of ranks floor(0.98 (n - 1)) and the next,
 *     found exactly), M~ = M (1 - clip((max(d_min - D, 0) + max(D - d_max,
 *     0)) / max(d_far - d_max, 1e-6), 0, 1)).
 * M is the mask probability (binary16, FP32, or the sigmoid of FP32 logits).
 * Non-finite depth means no surface: M~ = 0 there, and such pixels take no
 * part in min, max or the percentile; prompts / the centre at non-finite
 * depth are skipped; with none left (band) or max == min (min-max) the
 * weight is 1 on finite pixels.
 */
#define DIVAS_MAX_PROMPTS 15
enum { DIVAS_WEIGHT_NERF_MINMAX = 1, DIVAS_WEIGHT_GS_BAND = 2 };

typedef struct {
    const float* depth;   /* device H x W FP32 depth (D_exp or D_med), row-major          */
    const void* mask;     /* device H x W mask of mask_type                               */
    float* out;           /* device H x W FP32: the weighted mask (caller-owned)          */
    int32_t mask_type;    /* DIVAS_MASK_*                                                 */
    int32_t W, H;
    int32_t n_prompts;    /* GS_BAND: 0..DIVAS_MAX_PROMPTS positive prompts               */
    int32_t prompt_xy[2 * DIVAS_MAX_PROMPTS]; /* (x, y) pixel of each prompt, in frame    */
} divas_weight_view;

/* Weight n_views (1..DIVAS_MAX_VIEWS_PER_CALL) masks in `mode` on `stream`
 * (one launch per pass for all views; scratch in the context grows on demand
 * like the tuple scratch).  stats_out (device, nullable): n_views x 4 floats,
 * (min D, max D, n_finite, 0) for NERF_MINMAX, (d_min, d_max, d_far,
 * n_finite) for GS_BAND, NaN where undefined.  DIVAS_E_INVALID before any
 * launch: NULL rasters, bad sizes or mask_type, prompts outside the view. */
divas_status divas_depth_weight(divas_ctx* ctx, const divas_weight_view* views, int32_t n_views,
                                int32_t mode, float* stats_out, void* stream);

/* The depth-weighted masks of divas_depth_weight folded straight into the
 * fusion (Sec. 3.4, the weight applied where the vote reads the mask, Eq.
 * nerf-depthweight / Eqs. depthband, gs-bandpass, then Eqs. gs-depthweight
 * and vmask): views as for divas_fuse_add_views (1..32, each view's depth
 * raster D is also the depth the weight reads); every vote reads the mask
 * probability m at its pixel, gates m~ = m w(D) >= tau_mask and votes with
 * m~, w from the view's constants found by the same selection passes as
 * divas_depth_weight.  No weighted raster is written; the accumulators are
 * bitwise those of divas_depth_weight followed by divas_fuse_add_views of its
 * FP32 outputs.  prompts (host, n_views entries; may be NULL for
 * NERF_MINMAX): only n_prompts and prompt_xy are read (in frame of the
 * view).  stats_out: as for divas_depth_weight.  Errors: DIVAS_E_INVALID
 * before any launch (bad views, mode or prompts); DIVAS_E_STATE when the
 * selection scratch would have to grow inside a stream capture. */
divas_status divas_fuse_add_views_weighted(divas_ctx* ctx, const divas_view* views,
                                           const divas_weight_view* prompts, int32_t n_views,
                                           int32_t mode, float* stats_out, void* stream);

/*
 * Occupancy construction from 2DGS surfels (Sec. 3.5 "Occupancy by Morton-
 * scattered opacity"; Appendix "Occupancy grid construction"):
 *   Eq. scene-norm:  c = coordinate-wise median of the centres mu,
 *                    r_fg = P99(|mu - c|), b = max(ceil(pad r_fg), 1);
 *   Eq. voxel-size:  h = max(alpha_v s_bar, beta_v r_fg / g0), s_bar = the
 *                    median over surfels of their larger scale; g = the
 *                    smallest power of two >= 2 b / h, capped at g_max (h
 *                    raised to 2 b / g_max when the cap binds);
 *   the surfels inside the half-open cube c +- b scatter-add their opacity
 *   into voxel floor((mu - c + b) / h) of a g^3 density; occupied where
 *   density >= tau_tf.
 * Quantiles are the linear-interpolation ones of the finite values, found
 * exactly; distances are formed in FP64 and kept as FP32; the rules and the
 * voxel index are FP64.  The grid is linear (x fastest): origin = c - b,
 * edge h, side g (the fusion's plain grid).
 */
typedef struct {
    double alpha_v, beta_v; /* voxel-size weights (3, 1)                                   */
    double pad;             /* cube margin (1.05)                                          */
    int32_t g0, g_max;      /* reference and maximum grid side (256, 512; g_max a power of two <= 2048) */
    float tau_tf;           /* occupancy floor (0.5)                                       */
    int32_t reserved;
} divas_occupancy_params;

typedef struct {
    double c[3];      /* coordinate-wise median centre                      */
    double r_fg;      /* 99th-percentile radial distance                    */
    double b;         /* cube half-extent                                   */
    double s_bar;     /* median larger surfel scale                         */
    double h;         /* voxel edge                                         */
    double origin[3]; /* c - b: the grid's corner                           */
    int32_t g;        /* grid side                                          */
    int32_t pad;
} divas_scene_frame;

/* The paper's constants above (Table gs-hyperparams; g_max 512 as for LLFF). */
divas_occupancy_params divas_default_occupancy_params(void);

/* The frame from m surfels: mu (device m x 3 FP32 centres), scales (device
 * m x 2 FP32).  Synchronises `stream` (the grid side decides allocations).
 * DIVAS_E_INVALID: bad arguments or parameters, or no finite centre / scale. */
divas_status divas_scene_frame_from_gaussians(const float* mu, const float* scales, int64_t m,
                                              const divas_occupancy_params* params,
                                              divas_scene_frame* frame_out, void* stream);

/* The density (device g^3 FP32, 16-byte aligned, overwritten) and the dense
 * occupancy prior occ_out (device g^3 uint8, 4-byte aligned: 1 where density
 * >= tau_tf) of m surfels (mu as above, alpha device m FP32 opacities) in a
 * frame, on `stream`.  Density sums are FP32 atomics (their order varies). */
divas_status divas_occupancy_from_gaussians(const float* mu, const float* alpha, int64_t m,
                                            const divas_scene_frame* frame, float tau_tf,
                                            float* density, uint8_t* occ_out, void* stream);

/*
 * Voxel-to-surfel mapping for 2DGS, Passes 1-3 (Sec. 3.6 "Voxel-to-Surfel
 * Mapping and Aggregation"; Algorithm "Voxel-to-Surfel Mapping for 2DGS"):
 *   Pass 1 (Eq. pass1): F1 = the seg bit of the cell holding the centre (the
 *     context's seg bitfield of the last finalize, as divas_label_points);
 *   Pass 2 (Eqs. aspect, needle, pass-needle): a = max(s1, s2) / (min(s1, s2)
 *     + eps_aspect) (FP64, kept as FP32), tau_a = P99(a) found exactly,
 *     F2 = F1 and a <= tau_a;
 *   Pass 3 (Eqs. cov-atomics, kappa, final-F): in every view whose bit is set
 *     in the voxel's view mask (the context's vote bits), the tangent
 *     semi-axes t_k = s_k R[:, k] (k = 0, 1; R of the unit quaternion
 *     (w, x, y, z)), alpha_k = (pi(mu + t_k) - pi(mu - t_k)) / 2, the pixels
 *     whose centres lie in the 1-sigma box pi(mu) +- max(|alpha_0|, |alpha_1|)
 *     and pass the 3-sigma Cramer test (u^2 + v^2 <= 9 in tangent
 *     coordinates) count as visited, those with mask >= tau_m (logits:
 *     l >= logit(tau_m)) as foreground; F = F2 and, for some view,
 *     foreground >= tau_kappa max(visited, 1); kappa = the largest fraction.
 * A view counts only when the centre and the four tips are in front of
 * z_near.  Call after divas_fuse_finalize.
 */
typedef struct {
    float tau_m;       /* Pass 3 mask threshold (0.5)                  */
    float tau_kappa;   /* coverage threshold (0.5)                     */
    float eps_aspect;  /* aspect denominator guard (1e-8)              */
    int32_t reserved;
} divas_surfel_params;

/* The constants above (Table gs-hyperparams; eps_aspect is a reading). */
divas_surfel_params divas_default_surfel_params(void);

/* m surfels: mu (device m x 3), scales (device m x 2), quats (device m x 4,
 * (w, x, y, z)) FP32; n_views (0..DIVAS_MAX_VIEWS_PER_CALL) host cameras and
 * device masks of mask_type in the order of the views folded into the
 * context (view s is bit s).  Outputs (device, m each): f_out (final uint8),
 * f2_out (after Pass 2, nullable), kappa_out (FP32, nullable).  Scratch in
 * the context grows on demand (outside a stream capture). */
divas_status divas_surfel_labels(divas_ctx* ctx, const float* mu, const float* scales,
                                 const float* quats, int64_t m, const divas_camera* cams,
                                 const void* const* masks, int32_t mask_type, int32_t n_views,
                                 const divas_surfel_params* params, uint8_t* f_out,
                                 uint8_t* f2_out, float* kappa_out, void* stream);

/* The back-projected overlay of a view (Sec. 3.7 "Iterative Mask
 * Propagation": the fused 3D mask shown on the next view): out[y W + x] =
 * the seg bit of the cell holding the pixel centre (x + 1/2, y + 1/2)
 * unprojected at its planar depth (device H x W FP32), 0 where the depth is
 * not finite and positive or the point is outside the grid (device H x W
 * uint8).  Uses the seg bitfield of the last finalize. */
divas_status divas_overlay(divas_ctx* ctx, const divas_camera* cam, const float* depth,
                           uint8_t* out, void* stream);

/* Pass 1 labels (Eq. pass1): labels_out[i] = seg bit of the voxel containing
 * point i (device n x 3 float32), 0 outside the grid (half-open box), for NaN,
 * or for unoccupied voxels.  Uses the seg bitfield of the last finalize. */
divas_status divas_label_points(divas_ctx* ctx, const float* xyz, int64_t n, uint8_t* labels_out,
                                void* stream);

/* W = Z = bits = 0 and view count 0 (the active list is kept). */
divas_status divas_fuse_reset(divas_ctx* ctx, void* stream);

/* Wait for the context's queued work and report device-side errors. */
divas_status divas_fuse_sync(divas_ctx* ctx, void* stream);

/* Number of active voxels (host value; exact after init, capacity-bounded after
 * set_occupancy until the next synchronising call). */
int64_t divas_fuse_n_active(const divas_ctx* ctx);

/* Number of views folded in so far. */
int32_t divas_fuse_n_views(const divas_ctx* ctx);

/* Device n_active x 3 int32 (i, j, k) of the active list, in its order. */
divas_status divas_fuse_active_coords(divas_ctx* ctx, int32_t* coords_out, void* stream);

/* Export / import the accumulator state (checkpoint, eviction): device arrays
 * of n_active float32 W, float32 Z and uint32 bits, in active-list order. */
divas_status divas_fuse_export_state(divas_ctx* ctx, float* W_out, float* Z_out,
                                     uint32_t* bits_out, void* stream);
divas_status divas_fuse_import_state(divas_ctx* ctx, const float* W_in, const float* Z_in,
                                     const uint32_t* bits_in, int32_t n_views, void* stream);

/*
 * Adjoint of the fusion for a voxel-space cotangent (derived from Eq.
 * gs-depthweight and Eq. compact-fusion with the gates held fixed):
 *   dP/dm = w/Z, dP/dw = (m - P)/Z, dw/dD = w 2 alpha1 e / Delta^2,
 *   dm/dl = m (1 - m) for logit masks (1 for probability masks).
 * grad_score: device float32 dL/dP, dense g^3 (dense kind) or n_active
 * (sparse kind).  views: the same views, in the same order, that were folded
 * in (view k of the call is view k of the context).  grad_mask[k] and
 * grad_depth[k]: device float32 H x W rasters, accumulated into (atomic adds;
 * the caller zeroes them); either array of pointers, or any entry, may be
 * NULL to skip it.  Projections are recomputed per view; W and Z come from
 * the context, so call after the views were folded in.
 */
divas_status divas_fuse_backward(divas_ctx* ctx, const divas_view* views, int32_t n_views,
                                 const float* grad_score, float* const* grad_mask,
                                 float* const* grad_depth, void* stream);

/* Test hook: out_nr[i] = the projection's reciprocal of x[i] (hardware
 * approximation + one Newton-Raphson step), out_ieee[i] = the correctly
 * rounded reciprocal (device n floats each). */
divas_status divas_debug_rcp(const float* x, int64_t n, float* out_nr, float* out_ieee,
                             void* stream);

/* Test hook: the two integral images the depth-tuple mode builds per view, of
 * one W x H uint16 raster n_samp (device, row-major) into caller buffers s1
 * (uint32) and s2 (uint64), each (H + 1) x (W + 1) row-major with a zero
 * first row and column: s1[y][x] = sum of n over rows < y and columns < x
 * (mod 2^32), s2 the same of n^2 (mod 2^64).  Synchronises the stream. */
divas_status divas_debug_integral_images(const uint16_t* n_samp, int32_t W, int32_t H,
                                         uint32_t* s1, uint64_t* s2, void* stream);

/* Test hook: pixel index iy*W + ix that each active voxel projects to in a
 * camera, or -1 when it is behind z_near or out of frame (device n_active int32). */
divas_status divas_debug_project(divas_ctx* ctx, const divas_camera* cam, int32_t* pix_out,
                                 void* stream);

/*
 * Batched sessions: fold the views of many contexts (uneven grid sizes, kinds
 * and view counts) in ONE persistent launch, then finalize and label all of
 * them in one launch each.  Work items are (context, tile of its active
 * list), taken dynamically by the CTAs; each context's result is bitwise
 * identical to what its own add_views + finalize + label_points would give.
 *
 * Usage per batch: divas_batch_queue for each context (at most once per
 * batch, 1..32 views each), divas_batch_fuse, divas_batch_finalize (which
 * clears the queue).  A dry run (dry_run != 0) computes into batch scratch
 * and leaves the contexts untouched: it exists to time schedules (autotuning);
 * its first use allocates that scratch.  The batch stages descriptors in
 * pinned host memory (double-buffered) and copies them with one
 * cudaMemcpyAsync per call, so a fused-and-finalized batch can be captured in
 * a CUDA graph (the graph's copy keeps reading that staging buffer on every
 * replay, so a captured batch object must not be reused while the graph
 * lives).  fuse and finalize must run on the same stream.  The contexts of one
 * batch must not be used by other calls between queue and finalize.
 */
typedef struct divas_batch divas_batch;

typedef struct {
    int32_t threads;           /* 64, 128 or 256 per CTA */
    int32_t voxels_per_thread; /* 1, 2 or 4 voxels folded together per thread */
    int32_t ctas_per_sm;       /* persistent grid = SMs x ctas_per_sm (1..32) */
    int32_t tile;              /* voxels per work item, a multiple of threads x voxels_per_thread */
} divas_schedule;

divas_status divas_batch_create(divas_batch** out, int32_t max_sessions, int32_t max_views);
divas_status divas_batch_queue(divas_batch* b, divas_ctx* ctx, const divas_view* views,
                               int32_t n_views);
divas_status divas_batch_fuse(divas_batch* b, const divas_schedule* sched, int32_t dry_run,
                              void* stream);
/* score_out[k] / xyz[k] / n_pts[k] / labels_out[k] for the k-th queued context
 * (arrays and entries nullable): as divas_fuse_finalize's score_out and
 * divas_label_points.  flags: 0 or DIVAS_KEEP_ZEROS (the dense score_out
 * buffers already hold zeros for their unoccupied voxels: not refilled). */
divas_status divas_batch_finalize(divas_batch* b, float* const* score_out, const float* const* xyz,
                                  const int64_t* n_pts, uint8_t* const* labels_out, uint32_t flags,
                                  void* stream);
divas_status divas_batch_clear(divas_batch* b);
int32_t divas_batch_size(const divas_batch* b);
const char* divas_batch_last_error(const divas_batch* b);
void divas_batch_destroy(divas_batch* b);

/*
 * Allocation-free one-shot fusion of a dense prior: occupancy gate and active
 * list, all views, normalisation and consensus, in one call that allocates
 * nothing.  The paper has no counterpart: this exists for callers that must
 * not allocate device memory while they run, such as a per-frame plug-in
 * inside a host application that owns all GPU memory, where a cudaMalloc would
 * synchronise the device and stall the frame.
 *   grid: kind 0, not contracted, at most 64^3 cells (larger -> DIVAS_E_INVALID).
 *   occ_dense, views: as for divas_fuse_init / divas_fuse_add_views (1..32 views).
 *   score_out: device float32 g^3 (dense scores, 0 for unoccupied); nullable.
 *   seg_bits_out: device uint32 ceil(g^3/32) words; nullable.
 * Results equal divas_fuse_init + divas_fuse_add_views + divas_fuse_finalize.
 * Scratch lives in one device array of the library (about 4.3 MB, reserved on
 * every GPU that loads the library until exit) shared by all calls: calls that
 * overlap on the GPU race.  The first call on a device looks up that array's
 * address (once per device, with the device current); make it before any
 * stream capture.  Errors: DIVAS_E_INVALID before any launch for the same
 * invalid grids, parameters and cameras that divas_fuse_init and
 * divas_fuse_add_views reject (non-finite origin, intrinsics, R or t, NaN
 * thresholds, ...), for a side beyond 64, other grid kinds and bad views;
 * DIVAS_E_CUDA for a failed runtime call.  divas_noalloc_last_error returns
 * the message of this host thread's last failed call (thread-local, valid
 * until that thread's next call).
 */
divas_status divas_fuse_dense_noalloc(const divas_grid* grid, const uint8_t* occ_dense,
                                      const divas_view* views, int32_t n_views,
                                      const divas_params* params, float* score_out,
                                      uint32_t* seg_bits_out, void* stream);
const char* divas_noalloc_last_error(void);

void divas_fuse_destroy(divas_ctx* ctx);

/* Message of the last failing call on ctx (valid until the next call on ctx);
 * with ctx == NULL, the last failure of divas_fuse_init on this thread. */
const char* divas_last_error(const divas_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* DIVAS_FUSE_H */
