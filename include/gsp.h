/*
 * gsp.h -- C ABI of the GB300 stackless-BVH ray caster and stochastic progressive photon
 * mapping (SPPM) library.
 *
 * Method: T. Hachisuka, "Implementing a Photorealistic Rendering System using GLSL",
 * EGSR 2015. Sec. 2 (three-stage SPPM iteration), Sec. 3.1 / Fig. 3 (multiple-threaded BVH
 * traversal), Sec. 3.2 / Fig. 5 (PRNG), Sec. 3.3 (photon path regeneration), Sec. 3.4
 * (stochastic spatial hashing with random depth).
 *
 * Conventions shared by every entry point:
 *  - Every function returns gsp_status: 0 on success, a negative code otherwise. Nothing
 *    throws across the ABI. gsp_status_string() gives a static description.
 *  - Handles (gsp_context, gsp_scene, gsp_sppm) are opaque, owned by the library, and freed by
 *    the matching *_destroy call: renderers before their scene, scenes before their context (a
 *    handle keeps a pointer to its parent). A handle is not thread-safe; use one per host thread.
 *  - Host arrays ("h_" or documented as host) are read during the call and not retained.
 *  - Device arrays ("d_") are borrowed, caller-owned, contiguous, 16-byte aligned device
 *    memory on the context's device. They must stay valid until the stream work that uses
 *    them has completed.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy default stream. Device
 *    work is asynchronous on that stream. Kernels report faults they detect (a traversal that
 *    exceeds its step limit, an overflowing buffer) in a device status word; the next
 *    gsp_sppm_sync()/gsp_context_sync() returns the first such error.
 *  - Memory the library allocates itself (scene, BVH, SPPM state) lives in device memory of
 *    the context's device, sized at creation (a renderer makes both of its trace sets then). A
 *    few buffers are made on first use and kept: the per-stream buffers of host-buffer tracing,
 *    a batch's job tables; each entry point says so. Nothing is allocated between the launches
 *    of a pass.
 *  - Passes, batches and gradients use the handles' own extra streams internally; they are
 *    ordered after earlier work on `stream`, and later work on `stream` is ordered after them.
 *  - A CUDA error that earlier work left pending on the calling thread (the runtime's last error,
 *    which the library shares with every user of the same CUDA runtime) makes a call that launches
 *    device work return GSP_ERR_CUDA before it does anything, with gsp_last_error_message() naming
 *    the call and the error; it is neither discarded nor reported later as a failure of the call's
 *    own launches. A failing call consumes the error it reports, so the next call starts clean
 *    (a sticky error, one that ends the context, fails every later call).
 */
#ifndef GSP_H_
#define GSP_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t gsp_status;

enum {
    GSP_OK = 0,
    GSP_ERR_INVALID_ARG = -1,     /* a pointer, size or parameter is out of range */
    GSP_ERR_OOM = -2,             /* a device or host allocation failed */
    GSP_ERR_CUDA = -3,            /* a CUDA runtime call failed */
    GSP_ERR_TRAVERSAL_LIMIT = -4, /* a traversal exceeded its bound on box tests (corrupt links, or gsp_scene_set_step_limit) */
    GSP_ERR_TIMEOUT = -5,         /* a bounded device wait gave up */
    GSP_ERR_NOT_BUILT = -6,       /* the scene has no BVH yet (call gsp_build_bvh) */
    GSP_ERR_BAD_STATE = -7,       /* call order violated, e.g. render_grad before a forward */
    GSP_ERR_IO = -8,              /* checkpoint file could not be read or written */
    GSP_ERR_OVERFLOW = -9         /* a device buffer sized at creation overflowed */
};

typedef struct gsp_context gsp_context;
typedef struct gsp_scene gsp_scene;
typedef struct gsp_sppm gsp_sppm;

/* Material types. DIFFUSE: two-sided Lambertian with reflectance `albedo`; if `emission` is
 * non-zero it also emits Lambertian radiance `emission` from its front face (the side of
 * (v1-v0) x (v2-v0)). MIRROR: perfect reflection scaled by `albedo`. DIELECTRIC: smooth
 * interface of index `ior`, reflection or refraction picked with the exact unpolarised Fresnel
 * probability. EMITTER: one-sided Lambertian emitter of radiance `emission` that absorbs
 * everything it receives. */
enum { GSP_DIFFUSE = 0, GSP_MIRROR = 1, GSP_DIELECTRIC = 2, GSP_EMITTER = 3 };

typedef struct {
    int32_t type;
    float albedo[3];
    float emission[3];
    float ior;
} gsp_material; /* 32 bytes */

/* Pinhole camera: eye position, look-at point, up vector, full vertical field of view in
 * degrees, image size in pixels. Pixel (0, 0) is the top-left corner. */
typedef struct {
    float eye[3], look[3], up[3];
    float vfov_deg;
    int32_t width, height;
} gsp_camera; /* 48 bytes */

/* BVH build parameters (Sec. 3.1: top-down SAH build and threading on the host).
 *  bins           SAH bins per axis (default 16; 2..64)
 *  leaf_threshold a node with at most this many triangles becomes a leaf (default 4)
 *  max_leaf       hard cap on triangles per leaf (default 7, at most 7)
 *  link_sets      6 = multiple-threaded BVH (one hit/miss link set per ray direction class
 *                 +x,-x,+y,-y,+z,-z, Fig. 3); 1 = original threaded BVH (one fixed order). */
typedef struct {
    int32_t bins;
    int32_t leaf_threshold;
    int32_t max_leaf;
    int32_t link_sets;
} gsp_bvh_params;

typedef struct {
    int64_t nodes;        /* nodes in the tree (per link set) */
    int64_t leaves;
    int32_t depth;
    int32_t link_sets;
    double build_ms;      /* SAH build on the host */
    double thread_ms;     /* writing the hit/miss links of every link set on the host */
    int64_t device_bytes; /* node + triangle + shading bytes resident on the device */
} gsp_bvh_stats;

/* SPPM parameters.
 *  photons_per_pass  photon paths traced per pass (FULL_PATH) or photon threads (REGEN)
 *  table_size        hash table entries, a power of two; 0 = next_pow2(2 * photons_per_pass)
 *  seed              stream seed of the counter-based PRNG
 *  alpha             radius reduction parameter in (0, 1]
 *  r0                initial gather radius (world units, > 0)
 *  rr_continue       Russian-roulette continue probability at diffuse hits, in (0, 1]
 *  cell_h            hash cell edge; 0 = 2 * r0. Must be >= r0 / 4 (>= 2 * r0 in STOCHASTIC mode).
 *  eps               ray offset (tmin) of every secondary ray, world units
 *  photon_mode       GSP_FULL_PATH: whole photon paths each pass; GSP_REGEN: one bounce per
 *                    pass per thread, a thread starts a new path when its path ends (Sec. 3.3)
 *  hash_mode         GSP_EXACT: every photon within R is gathered; GSP_STOCHASTIC: one photon
 *                    survives per hash entry (minimum random depth), weighted by the entry's
 *                    photon count (Sec. 3.4)
 *  max_eye_depth     specular bounces followed by an eye path before it is dropped
 *  max_photon_depth  rays per photon path, at most 32
 *  scene_id          extra PRNG key so that batched scenes draw independent streams */
enum { GSP_FULL_PATH = 0, GSP_REGEN = 1 };
enum { GSP_EXACT = 0, GSP_STOCHASTIC = 1 };

typedef struct {
    int64_t photons_per_pass;
    int64_t table_size;
    uint64_t seed;
    float alpha, r0, rr_continue, cell_h, eps;
    int32_t photon_mode;
    int32_t hash_mode;
    int32_t max_eye_depth;
    int32_t max_photon_depth;
    uint32_t scene_id;
} gsp_sppm_params;

const char* gsp_status_string(gsp_status s);
/* Text of the last host-side error on the calling thread (CUDA message, build error), or "". */
const char* gsp_last_error_message(void);

/* ---- context ---------------------------------------------------------------------------- */

/* Creates a context on CUDA device `device` (the device is made current for the calling
 * thread). Owns a device status word used by every kernel of its scenes. */
gsp_status gsp_context_create(int32_t device, gsp_context** out);
void gsp_context_destroy(gsp_context* ctx);
/* Waits for all device work of the context and returns (then clears) the first device-side
 * error recorded by its kernels. */
gsp_status gsp_context_sync(gsp_context* ctx);

/* ---- PRNG (Sec. 3.2, Fig. 5) ------------------------------------------------------------- */

/* The renderer's random streams, written out: out[k * ndraw + j] = draw j of the stream keyed
 * by (seed, scene, domain, pass, d_ids[k]). A stream's four MLCG states are derived from the key
 * with SplitMix64 (s_i = 1 + 32-bit word i mod (m_i - 1)); each draw advances every state by
 * s' = a s mod m and returns fract(s0/m0 - s1/m1 + s2/m2 - s3/m3) evaluated left to right in
 * FP32 with round-to-nearest (1.0 is mapped to the largest float below 1). The renderer uses
 * domain 0 for eye paths (id = pixel) and 1 for photon paths (id = path or thread).
 * d_ids [n] uint64 device, d_out [n][ndraw] float device. */
gsp_status gsp_rng_fill(gsp_context* ctx, uint64_t seed, uint32_t scene, uint32_t domain, uint32_t pass,
                        const uint64_t* d_ids, int64_t n, int32_t ndraw, float* d_out, void* stream);

/* ---- scene (Sec. 3.1) -------------------------------------------------------------------- */

/* Uploads a triangle scene. Host inputs: verts [nv][3] float, tris [nt][3] int32 vertex
 * indices, tri_mat [nt] int32 material indices (NULL = all 0), mats [nmat], cam (NULL allowed
 * when only gsp_trace_closest_hit is used). Rejects non-finite vertices, out-of-range indices
 * and nmat outside 1..64 with GSP_ERR_INVALID_ARG. Zero-area triangles are kept; the
 * intersection test never reports them (determinant 0).
 * ctx == NULL makes a host-only scene that touches no GPU: it accepts gsp_build_bvh (which then
 * skips the upload), gsp_bvh_export and gsp_bvh_host_walk, and every device call rejects it. */
gsp_status gsp_scene_upload(gsp_context* ctx, const float* verts, int64_t nv, const int32_t* tris,
                            int64_t nt, const int32_t* tri_mat, const gsp_material* mats,
                            int32_t nmat, const gsp_camera* cam, gsp_scene** out);
void gsp_scene_destroy(gsp_scene* scene);

/* Replaces the scene's material table (same count, same validation as gsp_scene_upload).
 * Renderers created earlier keep the emitter table they were created with. */
gsp_status gsp_scene_set_materials(gsp_scene* scene, const gsp_material* mats, int32_t nmat);

/* Bounds the box tests of one ray's traversal (0 = the default, a few times the node count,
 * which only corrupt links can reach). A ray that reaches the bound ends early and the first
 * such event sets GSP_ERR_TRAVERSAL_LIMIT in the context's status word, which the next
 * gsp_context_sync / gsp_sppm_sync returns (and clears); nothing traps and the context stays
 * usable. Applies to launches made after the call (renderers read it per pass). For bounding
 * worst-case work, and for testing the failure path without corrupting a BVH. */
gsp_status gsp_scene_set_step_limit(gsp_scene* scene, int32_t max_box_tests);

/* Per-vertex shading data (Sec. 3.1: the threaded BVH's triangle record carries a normal and
 * texture coordinates at each vertex). Host arrays in upload order, copied:
 *   normals   [nv][3] per-vertex normals of any nonzero length, or NULL (face normals)
 *   texcoords [nv][2] per-vertex texture coordinates (s, t), or NULL (none)
 * At a hit the shading normal is the blend of the triangle's three vertex normals with the hit's
 * barycentric weights, normalised and turned into the geometric normal's hemisphere. It gives
 * the directions of mirror and dielectric bounces and the axis of a diffuse photon bounce's
 * cosine-distributed direction (a direction that points into the surface ends the photon path).
 * The geometric normal still decides the side a ray arrives from (emission, the photon
 * acceptance test). Both NULL removes the data. Takes effect for passes started afterwards (a
 * batch graph captured earlier keeps what it captured).
 * Errors: INVALID_ARG (non-finite value, zero normal); BAD_STATE (texcoords NULL while a
 * material has a texture); OOM; CUDA. */
gsp_status gsp_scene_set_attributes(gsp_scene* scene, const float* normals, const float* texcoords);

/* Albedo texture of a DIFFUSE material: rgb [height][width][3] factors (finite, >= 0) that
 * multiply the material's albedo. The lookup is bilinear with wrap-around at the blended texture
 * coordinates: texel (i, j) covers [i/width, (i+1)/width) x [j/height, (j+1)/height) and holds
 * its value at its centre. rgb NULL removes the texture. Host array, copied.
 * Errors: INVALID_ARG (material out of range or not DIFFUSE, width or height outside 1..16384,
 * more than 2^26 texels, a non-finite or negative value); BAD_STATE (the scene has no texture
 * coordinates); OOM; CUDA. */
gsp_status gsp_scene_set_texture(gsp_scene* scene, int32_t material, const float* rgb, int32_t width,
                                 int32_t height);

/* Builds the SAH BVH and its hit/miss links on the host (Sec. 3.1), packs them, and uploads
 * them to the device (replacing any previous BVH). params NULL = defaults. stats may be NULL. */
gsp_status gsp_build_bvh(gsp_scene* scene, const gsp_bvh_params* params, gsp_bvh_stats* stats);

/* Builds the BVH on the device instead (the paper's future work; Karras 2012): 30-bit Morton
 * codes of the triangle centroids, a stable radix sort, the radix tree's internal nodes found
 * independently, boxes bottom up, subtrees of at most max_leaf (1..7) triangles collapsed into
 * leaves, then the hit/miss links of link_sets (1 or 6) direction classes threaded in parallel
 * into the same packed layout gsp_build_bvh makes (and the child-pair layout of the stack
 * traversal). Every traversal entry point accepts the result; closest hits are the same, only
 * the work per ray differs (a Morton tree is not an SAH tree). stats.build_ms / thread_ms are
 * device times (codes to sizes; threading and layouts), excluding the upload of the vertex and
 * index arrays. Host copies are kept for gsp_bvh_host_walk / gsp_bvh_export. Device scenes only;
 * at most 2^28 triangles. */
gsp_status gsp_build_bvh_device(gsp_scene* scene, int32_t link_sets, int32_t max_leaf, gsp_bvh_stats* stats);

/* Closest-hit ray casting (Fig. 3): for each ray i, the triangle with the lexicographically
 * smallest (t, triangle index) among tmin < t < tmax, Moller-Trumbore in FP32; when the FP32
 * t of the winner may be inaccurate (origin far from the triangle compared with t, grazing
 * ray), its t and (u, v) are re-evaluated in FP64 from the exact vertices and rounded to FP32.
 *  d_rays [n][8] float: ox, oy, oz, tmin, dx, dy, dz, tmax (d need not be unit length)
 *  d_tri  [n] int32 out: triangle index in the uploaded order, -1 on a miss
 *  d_t    [n] float out: hit distance (in units of |d|), +inf on a miss
 *  d_uv   [n][2] float out or NULL: barycentrics (u, v) of the hit, 0 on a miss
 * Returns GSP_ERR_NOT_BUILT if the scene has no BVH. n == 0 is a no-op; n <= 2^31 - 1.
 * The scene keeps a list (8 bytes per ray) of hits whose t is re-evaluated in FP64; it is
 * allocated, after synchronising `stream`, the first time a call has more rays than any before. */
gsp_status gsp_trace_closest_hit(gsp_scene* scene, const float* d_rays, int64_t n, int32_t* d_tri,
                                 float* d_t, float* d_uv, void* stream);

/* Per-launch timing of the closest-hit kernel, for measuring it against its roofline (Fig. 3's
 * traversal alone). gsp_trace_time_launches(scene, n) makes n pairs of CUDA events (timing
 * enabled; any earlier pairs are destroyed; n = 0 just frees them, n <= 2^20); each of the next n
 * gsp_trace_closest_hit calls on the scene records one pair on its stream, immediately before and
 * after its traversal kernel, so the counter reset and the re-evaluation of flagged hits beside it
 * stay outside. The timed calls allocate nothing. gsp_trace_launch_times waits for the recorded
 * launches, writes the first min(count, capacity) durations in milliseconds to h_ms (host floats),
 * stores the number recorded in *count and starts recording again from the first pair.
 * GSP_ERR_INVALID_ARG on a host-only scene, n < 0 or n > 2^20. */
gsp_status gsp_trace_time_launches(gsp_scene* scene, int64_t n);
gsp_status gsp_trace_launch_times(gsp_scene* scene, float* h_ms, int64_t capacity, int64_t* count);

/* The same closest-hit query on HOST buffers (h_rays [n][8], h_tri [n], h_t [n], h_uv [n][2] or
 * NULL), synchronous. Page-locked buffers the device can address (cudaHostAlloc /
 * cudaHostRegister, e.g. pinned torch tensors; h_rays 16-byte aligned): the traversal reads the
 * rays from host memory itself, in two halves on two streams, and each half's results are copied
 * back while the other half is traced. Other buffers go in chunks of up to 2^20 rays through
 * page-locked staging buffers on three streams. The scene keeps per-stream device buffers (24
 * bytes per ray of a half or chunk, plus 32 + 48 bytes per ray of a chunk when staging),
 * allocated after a device synchronisation when first needed or outgrown. Results equal those
 * of gsp_trace_closest_hit. */
gsp_status gsp_trace_closest_hit_host(gsp_scene* scene, const float* h_rays, int64_t n, int32_t* h_tri,
                                      float* h_t, float* h_uv);

/* The same closest-hit query (same arguments, results and refinement) answered by a stack-based
 * near-first traversal of the same SAH tree, stored as child pairs (both children's boxes in one
 * 64-byte node): the kind of traversal the paper compares its stackless one with (Fig. 4; after
 * Aila & Laine 2009). For measuring the multiple-threaded BVH against it on this hardware.
 * GSP_ERR_INVALID_ARG if the tree is 64 or more levels deep (the per-ray stack holds 64). */
gsp_status gsp_trace_closest_hit_stack(gsp_scene* scene, const float* d_rays, int64_t n, int32_t* d_tri,
                                       float* d_t, float* d_uv, void* stream);

/* Instrumented host walk of the same threaded BVH (no GPU): per ray, the number of node
 * visits and triangle tests that the device traversal performs, and its closest hit.
 * Used to count the algorithmic bytes of a traversal. Host arrays; any output may be NULL. */
gsp_status gsp_bvh_host_walk(gsp_scene* scene, const float* h_rays, int64_t n, int32_t* h_tri,
                             float* h_t, int32_t* h_node_visits, int32_t* h_tri_tests);

/* Copies the packed BVH of link set `set` (0..link_sets-1) to host arrays (no GPU needed):
 *  h_nodes [nodes][8] float: min.xyz, miss link (int bits, -1 = none) | max.xyz, leaf word
 *          (int bits: bit 31 set = internal node, hit link = index + 1; otherwise
 *          triangle offset << 3 | triangle count, hit link = miss link)
 *  h_tris  [nt][12] float: v0.xyz, triangle index (int bits) | v1.xyz, 0 | v2.xyz, 0
 * Either pointer may be NULL; *nodes_out receives the node count. */
gsp_status gsp_bvh_export(gsp_scene* scene, int32_t set, float* h_nodes, float* h_tris,
                          int64_t* nodes_out);

/* ---- SPPM (Sec. 2, 3.3, 3.4) ------------------------------------------------------------- */

/* Creates a renderer over `scene` (which needs a camera, a BVH and at least one emitting
 * triangle). Allocates every device buffer a pass needs (pixel state, hit points, photon
 * records, hash table, sort scratch). */
gsp_status gsp_sppm_create(gsp_scene* scene, const gsp_sppm_params* params, gsp_sppm** out);
void gsp_sppm_destroy(gsp_sppm* r);

/* Runs `npasses` SPPM iterations on `stream`: eye pass (first non-specular hit per pixel,
 * emission seen directly), photon pass, hash-grid deposit, range query with the progressive
 * update N' = N + alpha M, R' = R sqrt((N + alpha M) / (N + M)), tau' = (tau + Phi) R'^2/R^2.
 * With npasses >= 2, the passes are traced on two streams of the renderer's own, alternating
 * between two sets of trace buffers and queues (with stochastic hashing, two tables; all made by
 * gsp_sppm_create, nothing is allocated during a pass): pass i + 1 is traced while the last paths
 * of pass i are still being traced and while pass i is deposited and gathered on `stream`; the
 * result equals npasses single-pass calls bit for bit. */
gsp_status gsp_sppm_pass(gsp_sppm* r, int32_t npasses, void* stream);

/* Execution tuning of the passes. eye_steps / photon_steps: wavefront steps (closest hit of a
 * compacted ray queue, then shading that pushes continuing paths to the next queue) before one
 * persistent kernel finishes the remaining eye and photon paths lane by lane; default 0 and 0.
 * Results do not depend on them.
 * refine_factor: 0 (default) = every wavefront hit takes its distance from the triangle's plane
 * in double-float arithmetic, as the persistent kernel's hits always do; > 0 = only hits whose
 * estimated FP32 error amplification exceeds it take an FP64 distance (trades hit-distance
 * accuracy for time).
 * gather_lanes: lanes that share one hit point's exact range query (1, 4, 8 or 16; 0 = keep);
 * the default at creation is 16 for images under 65,536 pixels and 8 from there on. Changes only
 * the order in which a pixel sums its photons.
 * traversal: GSP_TRAVERSAL_MTBVH (default) or GSP_TRAVERSAL_STACK for the persistent path kernel
 * (0 = keep); the closest hits, hence the results, are the same. The stack needs a tree less
 * than 64 levels deep (GSP_ERR_INVALID_ARG otherwise). */
#define GSP_TRAVERSAL_MTBVH 1 /* the path kernel follows the hit/miss links (the paper's traversal) */
#define GSP_TRAVERSAL_STACK 2 /* the path kernel walks the child-pair layout with a stack */
gsp_status gsp_sppm_tune(gsp_sppm* r, int32_t eye_steps, int32_t photon_steps, float refine_factor,
                         int32_t gather_lanes, int32_t traversal);

/* Writes the current estimate L = direct / P + tau / (pi R^2 N_e) to d_rgb [h][w][3] float. */
gsp_status gsp_sppm_image(gsp_sppm* r, float* d_rgb, void* stream);

/* Copies the per-pixel state to caller device arrays (any may be NULL): d_N [h*w],
 * d_R [h*w], d_tau [h*w][3], d_direct [h*w][3]. h_counts (host, may be NULL) receives
 * {passes, emitted paths N_e} after synchronising the stream. */
gsp_status gsp_sppm_state(gsp_sppm* r, float* d_N, float* d_R, float* d_tau, float* d_direct,
                          double* h_counts, void* stream);

/* The inverse of gsp_sppm_state: replaces the per-pixel progressive state (the N, R, tau update
 * of Sec. 2 and the direct term) from caller device arrays d_N [h*w], d_R [h*w] (each > 0),
 * d_tau [h*w][3], d_direct [h*w][3] (all required), and the pass count by `passes`; the next
 * pass continues from that state with pass index `passes` (the PRNG is keyed by it). For
 * restarting a render from a state computed elsewhere (a checkpoint written by other software,
 * or a reference renderer's state, so that one pass can be compared from identical state).
 * Whole photon paths only (GSP_ERR_BAD_STATE in the one-bounce mode, whose photon paths are not
 * part of this state, and after gsp_sppm_enable_grad). Every value is checked first: N finite
 * and >= 0, R finite in (0, r0], tau and direct finite and >= 0 (a larger radius would make the
 * exact gather visit cells without bound); otherwise GSP_ERR_INVALID_ARG and the renderer is
 * unchanged. Synchronises `stream` (to read the check). */
gsp_status gsp_sppm_set_state(gsp_sppm* r, const float* d_N, const float* d_R, const float* d_tau,
                              const float* d_direct, int64_t passes, void* stream);

/* Diagnostics of the last pass (host arrays, synchronises): number of photon deposits, and if
 * h_ids is not NULL (capacity given by the previous return value) their ids in ascending
 * order. Returns the count as a non-negative int64 or a negative gsp_status. */
int64_t gsp_sppm_last_deposits(gsp_sppm* r, uint32_t* h_ids, int64_t capacity);

/* Waits for the renderer's stream work and returns the first recorded device error. */
gsp_status gsp_sppm_sync(gsp_sppm* r);

/* Checkpoint: writes the renderer's progressive state (per-pixel N, R, tau, direct; the pass
 * count; in REGEN mode the per-thread photon paths; with gradients enabled the recorded radii
 * and flux sums) to a file. Synchronises the device. */
gsp_status gsp_sppm_save(gsp_sppm* r, const char* path);
/* Restores a checkpoint into a renderer created with the same scene and parameters (and, if the
 * checkpoint has gradient records, with gradients enabled for at least as many passes). The PRNG
 * is keyed by the pass index, so passes after a load give bit for bit the result of an
 * uninterrupted run. GSP_ERR_BAD_STATE if the parameters differ, GSP_ERR_IO if the file is
 * unreadable, short, followed by other data, or holds a pixel state no render reaches (the
 * values gsp_sppm_set_state checks); in each case the renderer is unchanged. */
gsp_status gsp_sppm_load(gsp_sppm* r, const char* path);

/* ---- many scenes per launch, CUDA graphs, autotuning ------------------------------------ */

typedef struct gsp_batch gsp_batch;

/* Groups renderers (of distinct scenes on one device; each renderer in at most one batch) so
 * that a pass of all of them runs as one CUDA graph: a branch per renderer, so the kernels of
 * small and large scenes overlap on the GPU. The graph is captured at the first gsp_batch_pass
 * and replayed for every pass; each branch reads its pass index from the device. Results are
 * those of gsp_sppm_pass on each renderer. Tuning changes (gsp_sppm_tune/autotune) made after the
 * first gsp_batch_pass do not reach the captured graph. A scene change that moves or resizes its
 * device data (a new BVH, new shading data, a step limit) makes the next gsp_batch_pass capture
 * again. The renderers must outlive the batch. */
gsp_status gsp_batch_create(gsp_sppm* const* renderers, int32_t n, gsp_batch** out);
void gsp_batch_destroy(gsp_batch* b);
/* Runs npasses passes of every renderer of the batch on `stream`. With one fused path launch
 * (gsp_batch_tune) and exact hashing in every renderer, pairs of passes run as a second graph of
 * two passes (captured at the first call that has a pair) in which the second pass is traced,
 * into the renderers' other trace sets, beside the first; results are unchanged. */
gsp_status gsp_batch_pass(gsp_batch* b, int32_t npasses, void* stream);

/* fused = 1: each batch pass runs the eye and photon fronts of all renderers in parallel
 * branches, then ONE persistent launch that finishes every renderer's eye and photon paths
 * (work items from all scenes in one queue: a warp's chunk names its renderer), then the
 * deposits and gathers in parallel branches (default). fused = 0: a path launch per renderer
 * inside its branch. Results are the same (bit for bit). Takes effect at the next pass (the graph
 * is captured again). */
gsp_status gsp_batch_tune(gsp_batch* b, int32_t fused);

typedef struct {
    int32_t eye_steps, photon_steps; /* chosen wavefront steps */
    float cell_h;                    /* chosen hash cell edge (exact mode) */
    float ms_per_pass;               /* its measured time per pass */
    float first_ms_per_pass;         /* time of the renderer's settings before tuning */
    int32_t candidates;              /* settings timed */
    int32_t gather_lanes;            /* chosen lanes per hit point in the exact gather (1, 4, 8, 16) */
    int32_t traversal;               /* chosen path-kernel traversal (GSP_TRAVERSAL_*) */
    int32_t fused;                   /* batch: 1 = one fused path launch for all renderers */
} gsp_tune_result;

/* Times candidate execution settings that leave the estimate unchanged, each from a fresh state
 * for trial_passes passes (after one untimed pass) on a temporary renderer over the same scene
 * (the renderer's own state is not touched), and applies the fastest: first the eye and photon
 * wavefront steps (0-2 and 0, 1, 2, 4), then in exact mode the hash cell edge (2, 1.5, 1, 0.75
 * or 0.5 times r0; smaller cells scan fewer photons but more buckets), then the lanes that share
 * one hit point's range query (1, 4, 8 or 16), then the path kernel's traversal (hit/miss links
 * or stack), replacing its current choice only for a gain above 3 %. Cell edge and lanes change
 * only the order in which a pixel sums its photons. out may be NULL. */
gsp_status gsp_sppm_autotune(gsp_sppm* r, int32_t trial_passes, gsp_tune_result* out);

/* Autotuning of a whole batch, before its first pass: times batch passes (one CUDA graph each)
 * under candidate settings applied to every renderer -- wavefront steps (eye 0-1, photon 0-2),
 * then the hash cell edge of the exact-mode renderers (2, 1.5, 1 or 0.75 times each renderer's
 * own r0; a stochastic renderer's edge is part of its estimate and stays), then lanes per hit point
 * in the exact gather (4, 8, 16), then the path kernel's traversal, then the other batch form
 * (gsp_batch_tune) with the steps searched again -- and keeps the fastest, replacing its current
 * choice only for a gain above 1 % (its trials are whole-batch passes, steady to well under that). Each candidate runs one
 * untimed and trial_passes timed passes, after which every renderer is back to its initial state,
 * so the renders that follow are those of untuned renderers (bit for bit for the steps and the
 * traversal; the cell edge and the lanes change only a pixel's summation order). GSP_ERR_BAD_STATE
 * if a renderer has run a pass, has gradients enabled or counts its work. out may be NULL (cell_h
 * reports renderer 0's). */
gsp_status gsp_batch_autotune(gsp_batch* b, int32_t trial_passes, gsp_tune_result* out);

/* ---- work counters (the algorithmic work of a pass, for rooflines) ------------------------- */

/* Indices of the work counts: eye rays traced (primary and specular continuations), photon rays
 * traced, node box tests, triangle tests (Fig. 3's two intersect calls), photon deposits, hit
 * points gathered, photons read by the gathers (candidates of the range query), hit points read
 * by the adjoint's photon-centric gather. */
#define GSP_WORK_EYE_RAYS 0
#define GSP_WORK_PHOTON_RAYS 1
#define GSP_WORK_NODE_VISITS 2
#define GSP_WORK_TRI_TESTS 3
#define GSP_WORK_DEPOSITS 4
#define GSP_WORK_HIT_POINTS 5
#define GSP_WORK_PHOTONS_SCANNED 6
#define GSP_WORK_HIT_POINTS_SCANNED 7
#define GSP_WORK_COUNTS 8

/* Counting the work of this renderer's passes (the paper has no counterpart: the counts give
 * the bytes and operations a pass must move, against which its time is held). Synchronises the
 * device, copies the counts accumulated since the previous call to h_counts [GSP_WORK_COUNTS]
 * (if not NULL), zeroes them, and switches counting on (on != 0) or off for the passes and
 * gradients that follow. Counting costs a few atomics per warp and per hit point; the estimate is
 * unchanged. It covers the persistent path kernels with the stackless traversal: GSP_ERR_BAD_STATE
 * if the renderer traces some bounces as wavefront steps or walks with a stack
 * (gsp_sppm_tune), and while it counts, gsp_sppm_tune to those settings, gsp_sppm_autotune,
 * gsp_batch_autotune and gsp_batch_pass with this renderer fail with GSP_ERR_BAD_STATE. */
gsp_status gsp_sppm_count_work(gsp_sppm* r, int32_t on, uint64_t* h_counts);

/* ---- gradient of an image loss (path-replay adjoint) ------------------------------------- */

/* Prepares gradients: every pass from now on records the radius each pixel gathered with and
 * the flux sum it gathered (20 bytes per pixel per pass, for at most max_passes passes; more
 * passes then fail with GSP_ERR_OVERFLOW) and the replay buffers are allocated. Call after gsp_sppm_create, before
 * the first pass. Needs photon_mode GSP_FULL_PATH, hash_mode GSP_EXACT, at most 64 materials and
 * exactly one emitting material (GSP_ERR_INVALID_ARG otherwise). */
gsp_status gsp_sppm_enable_grad(gsp_sppm* r, int32_t max_passes);

/* Gradient of a loss of the current image: d_dloss_dimg [h][w][3] float device is the loss's
 * gradient with respect to the image (L - target for 1/2 |L - target|^2). Outputs (float
 * device): d_grad_albedo [nmat][3], the derivative with respect to every material's albedo, and
 * d_grad_emission [3], with respect to the emitting material's emission. Russian roulette at a
 * constant probability makes the sampled paths, the gathered photon sets and the radii
 * independent of the albedos, so at fixed seeds the image is a polynomial in them; this is its
 * exact derivative. Each pass is replayed from its PRNG counters (no path is stored): its hit
 * points gather their weight into the photons they accepted (same test, recorded radius), and a
 * reverse walk along each photon path hands it to the albedos met before each deposit. Diffuse
 * albedos and the emission are differentiated; mirror and dielectric albedos are held constant
 * (their entries are 0), as are channels whose albedo is 0. The forward state is not changed. */
gsp_status gsp_render_grad(gsp_sppm* r, const float* d_dloss_dimg, float* d_grad_albedo,
                           float* d_grad_emission, void* stream);

/* ---- hash grid (the exact deposit of the SPPM pass as a standalone operation) ------------- */

/* Exact hash grid of a point set: the index the exact-mode deposit builds over a pass's photons
 * (Sec. 3.4 contrasts it with stochastic hashing). Per axis cell = floor(x / cell_h + 0.381966),
 * bucket = (ix*73856093 ^ iy*19349663 ^ iz*83492791) mod table_size (Teschner et al. 2003, 32-bit
 * wraparound; table_size a power of two <= 2^30). Points keep their input order inside a bucket.
 *  d_pos    [n] float4 device: x, y, z, (ignored); n <= 2^31 - 1
 *  d_order  [n] uint32 device out: point indices ordered by (bucket, input index)
 *  d_bstart [table_size + 1] uint32 device out: first position of each bucket in d_order;
 *           d_bstart[table_size] = n
 * Scratch (16 n bytes + about 0.6 MiB) lives on the context; it is allocated on first use and
 * reallocated (after synchronising `stream`) when a larger build needs more. */
gsp_status gsp_hash_grid_build(gsp_context* ctx, const float* d_pos, int64_t n, float cell_h,
                               int64_t table_size, uint32_t* d_order, uint32_t* d_bstart, void* stream);

/* The same hash-grid build without any device allocation (the paper has no counterpart: this
 * is a deployment variant). For callers that cannot allocate device memory: hosts whose device
 * memory belongs to another allocator or pool that forbids side allocations, plugins that are
 * handed fixed buffers, and real-time loops that must not block on cudaMalloc's implicit
 * synchronisation. Inputs and outputs are exactly those of gsp_hash_grid_build and are the
 * caller's buffers; no context is needed (the current device is
 * used). The scratch is a fixed array inside the library's device image (8.53 MiB, held on every
 * GPU that loads the library until the process exits), so:
 *  - n <= GSP_GRID_STATIC_MAX_POINTS and table_size <= GSP_GRID_STATIC_MAX_TABLE, otherwise
 *    GSP_ERR_INVALID_ARG with the limits in gsp_last_error_message();
 *  - the first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 *    that device current, and so does the first call after the current context has changed (a
 *    cudaDeviceReset, or another context made current through the driver API, loads the library's
 *    device image again); make such a call before any stream capture: during a capture it fails
 *    with GSP_ERR_BAD_STATE;
 *  - an error left pending by earlier CUDA work on the calling thread is reported (GSP_ERR_CUDA,
 *    message in gsp_last_error_message()) before anything is launched;
 *  - every call uses the same array, which keeps the previous call's contents (whatever must
 *    start at zero is cleared by the call itself); calls whose device work overlaps, on any
 *    streams, race on it and must be serialised by the caller.
 * No cudaMalloc, cudaFree or allocating library routine is called. */
#define GSP_GRID_STATIC_MAX_POINTS 524288
#define GSP_GRID_STATIC_MAX_TABLE 16777216
gsp_status gsp_hash_grid_build_static(const float* d_pos, int64_t n, float cell_h, int64_t table_size,
                                      uint32_t* d_order, uint32_t* d_bstart, void* stream);

/* ---- measurement --------------------------------------------------------------------------- */

/* Read bandwidth of the memory tier a buffer of `bytes` lives in (the paper has no counterpart:
 * this supplies the L2 peak against which the traversal of Sec. 3.1 is held). Allocates a
 * zero-filled device buffer of `bytes` (a multiple of 16, at least 16 KiB) on the context's device,
 * streams it once untimed, then `reps` times in one timed launch (16-byte loads that bypass L1;
 * one grid of 2,048 threads per SM), and frees it. *gbps = bytes * reps / time / 1e9. A buffer
 * well below the L2 size measures L2; one many times larger measures HBM. Synchronises the device.
 * GSP_ERR_OOM if the buffer does not fit. */
gsp_status gsp_measure_read_bandwidth(gsp_context* ctx, int64_t bytes, int32_t reps, double* gbps);

#ifdef __cplusplus
}
#endif

#endif /* GSP_H_ */
