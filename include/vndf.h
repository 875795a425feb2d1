/*
 * vndf.h -- C ABI of libvndf: spherical-cap sampling of GGX visible normals on
 * NVIDIA GB300 (sm_103a).
 *
 * Method: Dupuy & Benyoub, "Sampling Visible GGX Normals with Spherical Caps",
 * HPG 2023 (arXiv 2306.05044).  Every entry point below batches the paper's
 * per-sample problem "map two uniforms (u1, u2) in [0, 1), an incident
 * direction wi and roughnesses (alpha_x, alpha_y) to a microfacet normal wm"
 * (Sec. 2, "Importance Sampling") over n samples.
 *
 * Conventions shared by all entry points
 * --------------------------------------
 * - Arrays are structure-of-arrays float32 (or int32 where stated) in DEVICE
 *   memory, owned by the caller, and must stay valid until the work enqueued
 *   on `cuda_stream` has finished.  Element i of every array belongs to sample
 *   (or query) i.  Pointers must be 4-byte aligned; when every pointer of a
 *   call is 16-byte aligned the 128-bit vector path is taken, otherwise a
 *   scalar path.  Results never depend on the path, the launch shape or how a
 *   batch is split into calls.
 * - `cuda_stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *   are asynchronous and allocate no memory.  Outside stream capture the
 *   streaming and adjoint kernels are programmatic dependent launches: they
 *   may become resident while the work ahead of them on the stream drains,
 *   but wait for it to complete before they read or write any memory, so
 *   stream order holds exactly as for ordinary launches.
 * - n = 0 is a no-op that returns VNDF_OK without examining any pointer.
 * - Output arrays must not overlap input arrays or one another: a kernel may
 *   store an output before it has read every input it still needs (the
 *   double-float recomputation of an ill-conditioned sample rereads the
 *   sample's inputs after its FP32 result has been stored).  A call in which
 *   an output pointer equals an input pointer or another output pointer is
 *   rejected with VNDF_ERR_ARG; partial overlaps cannot be told from the
 *   pointers and give undefined results.  Inputs may share memory.
 * - Host-side argument errors return a negative VNDF_ERR_* code before any
 *   work is enqueued.  A failed launch, or a current device that cannot be
 *   queried (launch shapes are sized from its multiprocessor count), returns
 *   VNDF_ERR_CUDA.  Errors that happen while the kernel runs surface at the
 *   caller's next synchronisation.
 * - Fault injection, for testing a caller's error handling without making a
 *   GPU fail: when the environment variable VNDF_FAULT is "launch", "align"
 *   or "workspace", optionally followed by "@" and an entry point's name
 *   (e.g. "launch@vndf_sample"), every GPU entry point (or only the named
 *   one) returns, after its argument checks and before it enqueues anything,
 *   VNDF_ERR_CUDA, VNDF_ERR_ALIGN or (entry points that take a workspace
 *   only) VNDF_ERR_WORKSPACE.  The variable is read on every call; unset or
 *   empty, it has no effect.
 * - Domain: wi.z > 0, alpha_x > 0, alpha_y > 0, all finite.  wi need not be
 *   unit length (the method is invariant to its scale).  A sample outside the
 *   domain raises no error: it returns wm = (0, 0, 1) and pdf = 0.
 * - Random numbers: when u1 and u2 are both NULL, the uniforms are drawn in
 *   the kernel from Philox4x32-10 (Salmon et al., SC'11) with key = seed and
 *   counter = (b mod 2^32, b >> 32, stream_id, 0), b = g >> 1, where
 *   g = counter_base + i is the global index of sample i (mod 2^64).  An even g
 *   takes words (0, 1) of its block, an odd g words (2, 3); the first word
 *   gives u1 and the second u2 as (word >> 8) * 2^-24.  u1 drives the azimuth
 *   and u2 the cap height, as in both samplers the paper prints.
 */
#ifndef VNDF_H
#define VNDF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define VNDF_OK 0
#define VNDF_ERR_NULL (-1)      /* a required pointer is NULL                        */
#define VNDF_ERR_SIZE (-2)      /* a size is negative or above its stated limit      */
#define VNDF_ERR_ALIGN (-3)     /* a pointer is not aligned to its element size      */
#define VNDF_ERR_METHOD (-4)    /* unknown sampling method                           */
#define VNDF_ERR_WORKSPACE (-5) /* workspace missing or smaller than required        */
#define VNDF_ERR_CUDA (-6)      /* a CUDA runtime call or kernel launch failed       */
#define VNDF_ERR_ARG (-7)       /* optional arguments given in an invalid combination */

/* ---- sampling methods ------------------------------------------------ */
/* The paper's sampler: half vector between wi and a point drawn uniformly on
 * the spherical cap z in (-wi.z, 1] (Sec. 3.3, proved in Sec. 3.2). */
#define VNDF_METHOD_SPHERICAL_CAP 0
/* The prior sampler of Heitz 2018 that the paper improves on: uniform point on
 * the projected cross section of the hemisphere (Sec. 2, step (2)). */
#define VNDF_METHOD_POLAR_DISK 1
/* The spherical-cap sampler on the extended domain: incident directions
 * below the horizon as well.  Sec. 3.2-3.3 and Eq. 4 never use wi.z > 0: for
 * every stretched direction i with i.z > -1 the cap z in (-i.z, 1] and
 * sigma_std = (1 + i.z)/2 stay valid, and the samples are the normals with
 * wm.z > 0 that face wi, distributed as max(0, wi.wm) D(wm) / sigma(wi) with
 * sigma(wi) = (|M^-1 wi| + wi.z)/2 for unit wi (the projected area of the
 * microsurface).  Random walks on a microsurface meet such directions.  The
 * paper states the method for the upper hemisphere only; this extension is a
 * reading of it.  Domain: alpha_x, alpha_y > 0, all finite, and
 * 1 + i.z >= 2^-40 (i at least about 1.4e-6 rad from straight down); outside
 * it the usual fallback.  For wi.z > 0 results equal VNDF_METHOD_SPHERICAL_CAP
 * bit for bit.  Accepted by vndf_sample; its density at a given normal is
 * vndf_pdf_extended and its adjoint vndf_sample_backward_extended. */
#define VNDF_METHOD_SPHERICAL_CAP_EXTENDED 2

/* Version of this ABI; bumped on any incompatible change. */
int vndf_abi_version(void);

/* Static, NUL-terminated description of a status code (never NULL). */
const char *vndf_status_string(int status);

/* Whether the current CUDA device can dereference p: 1 for device or managed
 * memory and for page-locked host memory mapped into the device's address
 * space at the same address (on NVLink-C2C systems such host buffers can be
 * passed to every entry point directly, and the kernels then read and write
 * host memory without staging copies); 0 otherwise (including NULL and
 * ordinary pageable host memory); VNDF_ERR_CUDA if the query fails. */
int vndf_pointer_device_accessible(const void *p);

/*
 * vndf_rng_uniform -- the uniforms (u1, u2) that sample i would draw in
 * Philox mode (see "Random numbers" above; the paper only requires u in
 * [0, 1), Sec. 2).  Values lie in [0, 1 - 2^-24] and are exact float32.
 *   n        number of samples (0 <= n < 2^62); n = 0 is a no-op.
 *   u1, u2   outputs, n floats each (device).
 * Returns VNDF_OK, VNDF_ERR_NULL, VNDF_ERR_SIZE, VNDF_ERR_ALIGN, VNDF_ERR_ARG
 * (u1 == u2) or VNDF_ERR_CUDA.
 */
int vndf_rng_uniform(int64_t n, uint64_t seed, uint64_t counter_base, uint32_t stream_id,
                     float *u1, float *u2, void *cuda_stream);

/*
 * vndf_sample -- draw wm for each sample and, optionally, its density.
 * Sec. 2 steps (1)-(3): stretch wi by M^-1 = diag(alpha_x, alpha_y, 1) and
 * normalise; sample the hemisphere (method); unstretch by M^-T and normalise.
 * With VNDF_METHOD_SPHERICAL_CAP step (2) is the paper's Sec. 3.3 sampler.
 * The density is the GGX VNDF of Eq. 1,
 *   pdf = G1(wi) max(0, wi.wm) D(wm) / wi.z      (D, G1 as in App. A),
 * evaluated from the sampler's intermediate vectors rather than from the
 * rounded wm, so it stays accurate at small roughness.
 *   n                  number of samples (0 <= n < 2^62).
 *   wi_x, wi_y, wi_z   incident direction, pointing away from the surface.
 *   alpha_x, alpha_y   roughness; alpha_y = NULL means isotropic (alpha_y = alpha_x).
 *   u1, u2             explicit uniforms in [0, 1), or both NULL for in-kernel Philox.
 *   seed, counter_base, stream_id   Philox parameters (ignored with explicit u).
 *   method             VNDF_METHOD_SPHERICAL_CAP, VNDF_METHOD_POLAR_DISK or
 *                      VNDF_METHOD_SPHERICAL_CAP_EXTENDED.
 *   wm_x, wm_y, wm_z   outputs: unit microfacet normal.
 *   pdf                output density (solid angle of wm), or NULL to skip it.
 * Returns VNDF_OK or a negative VNDF_ERR_* code (NULL, SIZE, ALIGN, METHOD, ARG, CUDA).
 */
int vndf_sample(int64_t n,
                const float *wi_x, const float *wi_y, const float *wi_z,
                const float *alpha_x, const float *alpha_y,
                const float *u1, const float *u2,
                uint64_t seed, uint64_t counter_base, uint32_t stream_id,
                int method,
                float *wm_x, float *wm_y, float *wm_z, float *pdf,
                void *cuda_stream);

/*
 * vndf_rescue_count -- how many of these samples vndf_sample recomputes in
 * double-float.  The FP32 half vector h = c + i of the cap sampler (Sec. 3.3)
 * sums O(1) terms whose rounding the unstretch divides by |v|; vndf_sample
 * flags the samples whose condition number exceeds 24 and recomputes them
 * (the paper's method is exact; this is how the library meets its accuracy
 * bound in FP32).  This diagnostic runs the same per-sample function and
 * condition test on the same arguments as vndf_sample, discards the results
 * and writes the number of flagged samples, so a caller can see how often the
 * slow path runs on its inputs.  Arguments as for vndf_sample, plus:
 *   count    output, one unsigned 64-bit integer in device memory (8-byte
 *            aligned), set to 0 and then to the count; 0 for the prior sampler,
 *            which has no such path.
 * Returns VNDF_OK or a negative VNDF_ERR_* code (NULL, SIZE, ALIGN, METHOD, ARG, CUDA).
 */
int vndf_rescue_count(int64_t n,
                      const float *wi_x, const float *wi_y, const float *wi_z,
                      const float *alpha_x, const float *alpha_y,
                      const float *u1, const float *u2,
                      uint64_t seed, uint64_t counter_base, uint32_t stream_id,
                      int method, unsigned long long *count, void *cuda_stream);

/*
 * vndf_sample_reflection -- sample a reflected direction from the GGX
 * microfacet BRDF through the spherical-cap VNDF sampler (App. A, "Importance
 * Sampling Using the GGX VNDF"): wm is drawn exactly as vndf_sample draws it
 * (Sec. 2, Sec. 3.3), wi is reflected about it, wo = 2 (wi.wm) wm - wi
 * (Eq. reflect), and the outputs are
 *   pdf    = G1(wm, wi) D(wm) / (4 cos theta_i), the density of wo (App. A),
 *   weight = f_r(wo, wi) |cos theta_o| / pdf = F(wi.wm) G2 / G1(wi), the
 *            Monte Carlo weight of Eq. rendering_mc for unit radiance, with the
 *            height-correlated G2 of App. A and Schlick's Fresnel
 *            F0 + (1 - F0)(1 - wi.wm)^5; 0 when wo is below the surface.
 * wi.wm and the pdf are evaluated from the sampler's hemisphere vectors, so
 * they stay accurate next to the visibility boundary.
 *   n, wi_*, alpha_*, u1, u2, seed, counter_base, stream_id   as in vndf_sample.
 *   f0                 Schlick reflectance at normal incidence.
 *   wo_x, wo_y, wo_z   output reflected direction (unit).
 *   pdf, weight        outputs (each may be NULL to skip).
 * Out-of-domain samples give wo = (0, 0, 1), pdf = 0, weight = 0.
 * Returns VNDF_OK or a negative VNDF_ERR_* code (NULL, SIZE, ALIGN, ARG, CUDA).
 */
int vndf_sample_reflection(int64_t n,
                           const float *wi_x, const float *wi_y, const float *wi_z,
                           const float *alpha_x, const float *alpha_y,
                           const float *u1, const float *u2,
                           uint64_t seed, uint64_t counter_base, uint32_t stream_id,
                           float f0,
                           float *wo_x, float *wo_y, float *wo_z, float *pdf, float *weight,
                           void *cuda_stream);

/*
 * vndf_pdf -- GGX VNDF density of given normals (Eq. 1, written through the
 * App. A forms of D and G1):
 *   pdf = 2 max(0, wi.wm) / (pi alpha_x alpha_y (|M^-1 wi| + wi.z) Q^2),
 *   Q   = wm.x^2/alpha_x^2 + wm.y^2/alpha_y^2 + wm.z^2,
 * which is G1(wi) max(0, wi.wm) D(wm) / wi.z for unit wm.  wm is used as given
 * (unit length expected); wm.z <= 0 gives 0.  alpha_y = NULL means isotropic.
 * Returns VNDF_OK or a negative VNDF_ERR_* code (NULL, SIZE, ALIGN, ARG, CUDA).
 */
int vndf_pdf(int64_t n,
             const float *wi_x, const float *wi_y, const float *wi_z,
             const float *alpha_x, const float *alpha_y,
             const float *wm_x, const float *wm_y, const float *wm_z,
             float *pdf, void *cuda_stream);

/*
 * vndf_pdf_extended -- vndf_pdf on the domain of
 * VNDF_METHOD_SPHERICAL_CAP_EXTENDED (wi may lie below the horizon):
 *   pdf = max(0, wi.wm) D(wm) / sigma(wi),  sigma(wi) = (|M^-1 wi| + wi.z)/2
 * for unit wi (Eq. 1 with the projected area of Eq. 4 carried through M; it
 * equals the G1 form of vndf_pdf wherever wi.z > 0).  Same arguments, layout
 * and errors as vndf_pdf; inputs outside the extended domain, or wm.z <= 0,
 * give 0.
 */
int vndf_pdf_extended(int64_t n,
                      const float *wi_x, const float *wi_y, const float *wi_z,
                      const float *alpha_x, const float *alpha_y,
                      const float *wm_x, const float *wm_y, const float *wm_z,
                      float *pdf, void *cuda_stream);

/*
 * vndf_sample_hemisphere -- the spherical-cap sampler of Sec. 3.3 used on its
 * own: visible normals of the hemisphere configuration (D_std = 1/pi on the
 * upper hemisphere, Eq. 3) seen from direction wi.  Sec. 3.3 leaves the half
 * vector h = c + wi unnormalised because the GGX sampler normalises after
 * unstretching; here the output is h / |h|, the normalisation a stand-alone
 * use needs, and the density is Eq. 2,
 *   pdf = max(0, wi.wm) / (pi sigma_std(wi.z)),  sigma_std = (1 + wi.z)/2 (Eq. 4),
 * which equals |h| / (pi (1 + wi.z)) at the sample.  It is the GGX sampler
 * with alpha_x = alpha_y = 1 (where D = 1/pi) without the roughness streams.
 *   n                  number of samples (0 <= n < 2^62).
 *   wi_x, wi_y, wi_z   direction (any length; normalised internally); the
 *                      extended domain applies: 1 + wi.z/|wi| >= 2^-40, finite.
 *   u1, u2             explicit uniforms in [0, 1), or both NULL for in-kernel Philox.
 *   seed, counter_base, stream_id   Philox parameters (ignored with explicit u).
 *   wm_x, wm_y, wm_z   outputs: unit normal (wm.z > 0); (0, 0, 1) outside the domain.
 *   pdf                output density (solid angle), or NULL to skip it; 0 outside the domain.
 * Returns VNDF_OK or a negative VNDF_ERR_* code (NULL, SIZE, ALIGN, ARG, CUDA).
 */
int vndf_sample_hemisphere(int64_t n,
                           const float *wi_x, const float *wi_y, const float *wi_z,
                           const float *u1, const float *u2,
                           uint64_t seed, uint64_t counter_base, uint32_t stream_id,
                           float *wm_x, float *wm_y, float *wm_z, float *pdf,
                           void *cuda_stream);

/*
 * vndf_sample_backward -- reparameterised gradients of the spherical-cap
 * sampler and its fused pdf (vndf_sample with VNDF_METHOD_SPHERICAL_CAP):
 * the vector-Jacobian product of (wm, pdf) with respect to (wi, alpha_x,
 * alpha_y), with the uniforms u held fixed.  The paper gives the forward map
 * (Sec. 2 steps (1)-(3), Sec. 3.3, Eq. 1); this is its exact adjoint, computed
 * by recomputing the forward in registers (nothing is stored between calls).
 *   n, wi_*, alpha_*, u1, u2, seed, counter_base, stream_id
 *                       exactly as given to vndf_sample (same u for the same i).
 *   g_wm_x, g_wm_y, g_wm_z  adjoint of wm (all three NULL = zero).
 *   g_pdf               adjoint of pdf (NULL = zero).
 *   g_wi_x, g_wi_y, g_wi_z  outputs d/d wi (all three NULL = not written).
 *   g_alpha_x           output d/d alpha_x (NULL = not written); with an
 *                       isotropic call (alpha_y = NULL) it receives d/d alpha.
 *   g_alpha_y           output d/d alpha_y (NULL = not written; must be NULL
 *                       when alpha_y is NULL).
 * Samples outside the domain get zero gradients.  Because the sampler is
 * invariant to the scale of wi, g_wi . wi = 0 up to rounding.
 * Returns VNDF_OK or a negative VNDF_ERR_* code (NULL, SIZE, ALIGN, ARG, CUDA).
 */
int vndf_sample_backward(int64_t n,
                         const float *wi_x, const float *wi_y, const float *wi_z,
                         const float *alpha_x, const float *alpha_y,
                         const float *u1, const float *u2,
                         uint64_t seed, uint64_t counter_base, uint32_t stream_id,
                         const float *g_wm_x, const float *g_wm_y, const float *g_wm_z,
                         const float *g_pdf,
                         float *g_wi_x, float *g_wi_y, float *g_wi_z,
                         float *g_alpha_x, float *g_alpha_y,
                         void *cuda_stream);

/*
 * vndf_sample_backward_extended -- vndf_sample_backward for
 * VNDF_METHOD_SPHERICAL_CAP_EXTENDED (incident directions below the horizon
 * too; the extension is a reading of Sec. 3.2-3.3 and Eq. 4, see that method):
 * the same vector-Jacobian product of (wm, pdf), with the pdf of
 * vndf_pdf_extended, on the extended domain.  Same arguments, layout and
 * errors as vndf_sample_backward; samples outside the extended domain get
 * zero gradients.
 */
int vndf_sample_backward_extended(int64_t n,
                                  const float *wi_x, const float *wi_y, const float *wi_z,
                                  const float *alpha_x, const float *alpha_y,
                                  const float *u1, const float *u2,
                                  uint64_t seed, uint64_t counter_base, uint32_t stream_id,
                                  const float *g_wm_x, const float *g_wm_y, const float *g_wm_z,
                                  const float *g_pdf,
                                  float *g_wi_x, float *g_wi_y, float *g_wi_z,
                                  float *g_alpha_x, float *g_alpha_y,
                                  void *cuda_stream);

/* Device workspace (bytes) that vndf_sample_loss_backward needs for n samples:
 * one float per 128-sample group, one per segment of 2048 groups, and a
 * counter.  0 for n <= 0. */
size_t vndf_loss_workspace_bytes(int64_t n);

/*
 * vndf_sample_loss_backward -- fused forward, loss and adjoint for the
 * reparameterised objective
 *   loss = sum_i ( c_i . wm_i + log pdf_i )
 * over the spherical-cap samples of vndf_sample (Sec. 2, Sec. 3.3, Eq. 1):
 * writes the loss and its gradients with respect to wi and alpha in one pass
 * (g_wm = c and d loss / d log pdf = 1 per sample).  Samples outside the
 * domain contribute nothing and get zero gradients.
 *   c_x, c_y, c_z       per-sample weight vectors (device).
 *   g_wi_*, g_alpha_*   outputs as in vndf_sample_backward (NULL = skip).
 *   loss                output, one float (device).  It is summed per fixed
 *                       128-sample group, then per fixed segment of 2048
 *                       groups, then over the segments, each level in an
 *                       order that depends only on n, so it is
 *                       bit-reproducible for a given n.
 *   workspace           device scratch of >= vndf_loss_workspace_bytes(n)
 *                       bytes, owned by the caller; its contents on entry are
 *                       ignored.  Concurrent calls need separate workspaces.
 * Returns VNDF_OK or a negative VNDF_ERR_* code (NULL, SIZE, ALIGN, ARG,
 * WORKSPACE, CUDA).
 */
int vndf_sample_loss_backward(int64_t n,
                              const float *wi_x, const float *wi_y, const float *wi_z,
                              const float *alpha_x, const float *alpha_y,
                              const float *c_x, const float *c_y, const float *c_z,
                              const float *u1, const float *u2,
                              uint64_t seed, uint64_t counter_base, uint32_t stream_id,
                              float *g_wi_x, float *g_wi_y, float *g_wi_z,
                              float *g_alpha_x, float *g_alpha_y,
                              float *loss, void *workspace, size_t workspace_bytes,
                              void *cuda_stream);

/* Device workspace (bytes) for vndf_albedo_batched / vndf_albedo_autotune with
 * n_queries queries of at most max_samples_per_query samples each:
 * control words (item scan, counters) plus one float per 256-sample group
 * slot.  0 when n_queries <= 0 or when the batch exceeds the limits of
 * vndf_albedo_batched (max_samples_per_query > 2^30, or n_queries x
 * ceil(max_samples_per_query / 256) >= 2^31). */
size_t vndf_albedo_workspace_bytes(int32_t n_queries, int32_t max_samples_per_query);

/*
 * vndf_albedo_batched -- directional albedo of the GGX microfacet BRDF for a
 * ragged batch of queries, estimated in one persistent launch with the
 * spherical-cap VNDF sampler:
 *   E_q = (1/N_q) sum_j f_r(wo_j, wi_q) |cos theta_o| / PDF(wo_j),
 * the Monte Carlo estimator of App. A (Eq. rendering_mc with L = 1): wm_j is
 * sampled as in vndf_sample (Sec. 2, Sec. 3.3), wo_j is wi reflected about it
 * (Eq. reflect) and PDF = G1 D / (4 cos theta_i) (App. A).  f_r is the
 * Cook-Torrance BRDF of App. A with the height-correlated G2 and Schlick's
 * Fresnel F0 + (1 - F0)(1 - wi.wm)^5; terms with wo below the surface are 0.
 *   n_queries          number of queries (>= 0); 0 is a no-op.
 *   wi_*, alpha_*      per-query direction (upper hemisphere, any length) and
 *                      roughness; alpha_y = NULL means isotropic.  A query
 *                      outside the sampler's domain (wi.z <= 0, alpha <= 0,
 *                      non-finite) yields E_q = NaN.
 *   n_samples          per-query sample counts N_q (int32, device).  A count
 *                      outside [0, max_samples_per_query] yields E_q = NaN; a
 *                      count of 0 (in the domain) yields E_q = 0.
 *   max_samples_per_query  the bound the workspace was sized for (<= 2^30,
 *                      and n_queries x ceil(max_samples_per_query / 256)
 *                      < 2^31 so that every 256-sample group slot has an
 *                      int32 index; larger batches return VNDF_ERR_SIZE).
 *   f0                 Schlick reflectance at normal incidence.
 *   seed, counter_base, stream_id  Philox: query q draws from stream
 *                      stream_id + q, sample j from global index counter_base + j.
 *   E                  output, n_queries floats (device).
 *   workspace          device scratch of >= vndf_albedo_workspace_bytes(...)
 *                      bytes, 256-byte aligned, owned by the caller; contents on
 *                      entry are ignored.  Concurrent calls need separate
 *                      workspaces.
 *   config             NULL (use the configuration vndf_albedo_autotune picked
 *                      on this device, else a default) or three int32 on the
 *                      host: warps per CTA (1-20), 256-sample groups per work
 *                      item (1-256; each warp takes a contiguous run of whole
 *                      items, the runs of all warps within one item of each
 *                      other), CTAs per SM (1-32; capped at the number an SM
 *                      holds at once, so that every CTA starts immediately).
 * The summation order is fixed by the data (256-sample groups, then groups in
 * order), so E is bit-identical for every config, every split of the queries
 * into calls, and every replay of a captured CUDA graph.
 * Returns VNDF_OK or a negative VNDF_ERR_* code (NULL, SIZE, ALIGN, ARG,
 * WORKSPACE, CUDA).
 */
int vndf_albedo_batched(int32_t n_queries,
                        const float *wi_x, const float *wi_y, const float *wi_z,
                        const float *alpha_x, const float *alpha_y,
                        const int32_t *n_samples, int32_t max_samples_per_query,
                        float f0, uint64_t seed, uint64_t counter_base, uint32_t stream_id,
                        float *E, void *workspace, size_t workspace_bytes,
                        const int32_t *config, void *cuda_stream);

/*
 * vndf_albedo_autotune -- time vndf_albedo_batched on the given batch for a
 * fixed set of launch configurations (warps per CTA x groups per item x CTAs
 * per SM), remember the fastest for the current device (later calls with
 * config = NULL use it) and return it.  Synchronises `cuda_stream`; not for
 * use during stream capture.  Arguments as for vndf_albedo_batched (E is
 * overwritten with the batch result), plus:
 *   best_config        output, three int32 on the host (may be NULL).
 *   best_ms            output, best time in milliseconds (host, may be NULL).
 * Returns VNDF_OK or a negative VNDF_ERR_* code.
 */
int vndf_albedo_autotune(int32_t n_queries,
                         const float *wi_x, const float *wi_y, const float *wi_z,
                         const float *alpha_x, const float *alpha_y,
                         const int32_t *n_samples, int32_t max_samples_per_query,
                         float f0, uint64_t seed, uint64_t counter_base, uint32_t stream_id,
                         float *E, void *workspace, size_t workspace_bytes,
                         int32_t *best_config, float *best_ms, void *cuda_stream);

/*
 * vndf_albedo_set_config -- set the launch configuration that
 * vndf_albedo_batched (and its no-allocation variant) use on the current
 * device when called with config = NULL, as vndf_albedo_autotune does after
 * timing; NULL restores the default.  Lets a caller reuse a configuration it
 * tuned earlier (for instance one stored on disk by the Python binding's
 * autotune cache) without timing again.  The configuration only chooses the
 * launch shape: E is the same for every configuration.
 *   config   three int32 on the host (warps per CTA 1-20, groups per item
 *            1-256, CTAs per SM 1-32), or NULL.
 * Returns VNDF_OK, VNDF_ERR_ARG (a value out of range), VNDF_ERR_SIZE (a
 * device ordinal above 63) or VNDF_ERR_CUDA (no current device).
 */
int vndf_albedo_set_config(const int32_t *config);

/*
 * vndf_albedo_get_config -- the configuration a config = NULL call of
 * vndf_albedo_batched uses on the current device, written to three int32 on
 * the host.  Returns 1 when it was set (by vndf_albedo_autotune or
 * vndf_albedo_set_config), 0 when it is the default, VNDF_ERR_NULL or
 * VNDF_ERR_CUDA.
 */
int vndf_albedo_get_config(int32_t *config);

/* Device workspace (bytes) for vndf_fit_step: one float per texel. */
size_t vndf_fit_workspace_bytes(int32_t n_texels);

/*
 * vndf_fit_step -- one optimisation step of an anisotropic roughness map so
 * that the mean of its sampled visible normals matches a target map: the
 * reparameterised use of the sampler that its adjoint exists for.  Per texel
 * t, S = samples_per_texel normals are drawn with the spherical-cap sampler
 * (Sec. 2 steps (1)-(3), Sec. 3.3) from Philox stream stream_id + t at global
 * indices counter_base + (step - 1) S + j, so every step draws fresh samples;
 *   m_t  = (1/S) sum_j wm_tj,      loss = (1 / 3N) sum_t |m_t - target_t|^2
 * (N = n_texels_total, else T),
 * the gradient with respect to (alpha_x, alpha_y) goes through the adjoint of
 * vndf_sample_backward, and Adam (Kingma & Ba 2015, with bias correction at
 * the 1-based step) updates alpha, which is then clamped to
 * [alpha_min, alpha_max].  The paper defines the sampler only; this loop is
 * the library's use of it.
 *   n_texels, samples_per_texel   T >= 0 and 1 <= S <= 2^20.
 *   n_texels_total      size of the whole map when these T texels are one
 *                       part of it (0 = T).  The loss and its gradient are
 *                       normalised by it, so splitting a map into calls (one
 *                       per GPU, each with stream_id = its first texel) gives
 *                       the same updates, bit for bit, as one call over the
 *                       whole map, and the calls' losses add up to its loss.
 *                       Must be 0 or >= T.
 *   wi_*, target_*      per-texel incident direction and target mean (read).
 *   alpha_x, alpha_y    per-texel roughness (read and updated in place).
 *   adam_m_*, adam_v_*  Adam moments (read and updated; zero before step 1).
 *   step                one int64 in device memory: the number of completed
 *                       steps.  The call performs step *step + 1 and adds one
 *                       at the end, in stream order, so a CUDA graph that
 *                       captured this call advances on every replay.
 *   lr, beta1, beta2, eps, alpha_min, alpha_max   optimiser settings
 *                       (0 <= beta < 1, 0 < alpha_min <= alpha_max).
 *   loss                output, one float (device; NULL = skip): the loss at
 *                       the parameters before this step's update.
 *   workspace           device scratch of >= vndf_fit_workspace_bytes(T)
 *                       bytes (caller-owned; contents ignored on entry).
 * All sums run in a fixed order, so a run is bit-reproducible and resumable
 * from saved (alpha, moments, step).
 * Returns VNDF_OK or a negative VNDF_ERR_* code (NULL, SIZE, ALIGN, ARG,
 * WORKSPACE, CUDA).
 */
int vndf_fit_step(int32_t n_texels, int32_t n_texels_total, int32_t samples_per_texel,
                  const float *wi_x, const float *wi_y, const float *wi_z,
                  const float *target_x, const float *target_y, const float *target_z,
                  float *alpha_x, float *alpha_y,
                  float *adam_m_x, float *adam_m_y, float *adam_v_x, float *adam_v_y,
                  int64_t *step,
                  float lr, float beta1, float beta2, float eps, float alpha_min, float alpha_max,
                  uint64_t seed, uint64_t counter_base, uint32_t stream_id,
                  float *loss, void *workspace, size_t workspace_bytes, void *cuda_stream);

/*
 * vndf_microbench -- the paper's GPU benchmark protocol (Sec. 4, "GPU
 * Synthetic Benchmark": the GGX VNDF sampler called 64 times per lane) as a
 * kernel.  Each lane draws its incident direction and roughness in registers,
 * samples `samples_per_lane` normals with `method` and their fused pdf, and
 * writes the four sums (sum wm.x, sum wm.y, sum wm.z, sum pdf), so only
 * 16 bytes per lane reach memory and the time measures the sampler's
 * arithmetic.  Lane l's inputs come from Philox4x32-10 block
 * (l mod 2^32, l >> 32, 0xffffffff, 0) with key = seed, as 24-bit uniforms
 * v0..v3: cos(theta_i) = 1e-4 + (1 - 1e-4) v0, phi_i = 2 pi v1,
 * alpha_x = 1e-3^(1 - v2), alpha_y = 1e-3^(1 - v3).  Sample j of lane l uses
 * the vndf_sample layout with stream 0 and global index l * samples_per_lane + j.
 *   lanes              number of lanes (0 <= lanes < 2^40).
 *   samples_per_lane   1 .. 2^20 (the paper uses 64).
 *   precise            spherical cap only: nonzero runs the sampler exactly as
 *                      vndf_sample does (ill-conditioned samples recomputed in
 *                      double-float, every sample within 4e-6 rad of FP64);
 *                      0 runs the plain FP32 sampler, the accuracy class of
 *                      the prior sampler (which has no such path).
 *   sums               output, 4 floats per lane (device, 16-byte aligned).
 * Returns VNDF_OK or a negative VNDF_ERR_* code (NULL, SIZE, ALIGN, METHOD, CUDA).
 */
int vndf_microbench(int64_t lanes, int32_t samples_per_lane, int method, int precise, uint64_t seed,
                    float *sums, void *cuda_stream);

/*
 * vndf_cpu_sample -- the GGX VNDF sampler on the host CPU, for the paper's CPU
 * benchmark (Sec. 4, "CPU Synthetic Benchmark", which calls the sampler in a
 * loop).  An explicit host entry point, not a fallback of vndf_sample: all
 * pointers are HOST memory, uniforms are explicit, and the arithmetic is FP32
 * with the same rounding-aware formulas as the GPU kernels, vectorised by the
 * compiler and split over `threads` host threads (0 = all hardware threads).
 *   method             any VNDF_METHOD_* (the extended cap method as in
 *                      vndf_sample).
 *   precise            cap methods only: nonzero recomputes the samples whose
 *                      half vector is ill-conditioned (the condition test of
 *                      vndf_sample) in double precision, so that every sample
 *                      meets 4e-6 rad and 1e-5 relative (wi.z >= 1e-4, alpha
 *                      >= 1e-3), as vndf_sample does; 0 runs the plain FP32
 *                      sampler, the accuracy class of the prior sampler (about
 *                      1e-5 of samples beyond 4e-6 rad), which the paper's
 *                      benchmark times.  Ignored for the prior sampler.
 *   threads            host threads (0 = all hardware threads).
 * Results do not depend on the thread count.
 * Returns VNDF_OK or a negative VNDF_ERR_* code (NULL, SIZE, METHOD, ARG).
 */
int vndf_cpu_sample(int64_t n,
                    const float *wi_x, const float *wi_y, const float *wi_z,
                    const float *alpha_x, const float *alpha_y,
                    const float *u1, const float *u2, int method, int precise,
                    float *wm_x, float *wm_y, float *wm_z, float *pdf, int threads);

/* Size of the fixed device scratch array behind vndf_albedo_batched_noalloc:
 * 8 MiB.  A batch fits when vndf_albedo_workspace_bytes(n_queries,
 * max_samples_per_query) is at most this; 4096 queries of up to 65536 samples
 * each need about 4.03 MiB. */
#define VNDF_ALBEDO_NOALLOC_SCRATCH_BYTES (8u << 20)

/*
 * vndf_albedo_batched_noalloc -- vndf_albedo_batched for callers that cannot
 * allocate device memory or pass a workspace (for instance a renderer's frame
 * loop, where a cudaMalloc would synchronise the device, or a plugin that only
 * receives pointers from a host application that owns all device memory).
 * The paper has no counterpart; this is a deployment variant.
 * It allocates nothing: its scratch is a file-scope device array of
 * VNDF_ALBEDO_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds
 * until the process exits.  The caller still provides all inputs and the output
 * E, with the meaning and results of vndf_albedo_batched.
 *   - Batches whose vndf_albedo_workspace_bytes(n_queries,
 *     max_samples_per_query) exceeds the array are rejected with
 *     VNDF_ERR_SIZE before anything is enqueued.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress, with that device current) and caches it; make that
 *     first call before any stream capture.
 *   - All calls on a device share the one array.  Each call resets the parts it
 *     reads, but calls that overlap on the GPU (concurrent streams, or several
 *     host threads) race on it: order them on one stream.
 *   - The cached address belongs to the device's current context: after
 *     cudaDeviceReset (or anything else that destroys and recreates the
 *     primary context) it is stale, and the entry point must not be called
 *     again in that process.
 * Returns VNDF_OK or a negative VNDF_ERR_* code (NULL, SIZE, ALIGN, ARG, CUDA).
 */
int vndf_albedo_batched_noalloc(int32_t n_queries,
                                const float *wi_x, const float *wi_y, const float *wi_z,
                                const float *alpha_x, const float *alpha_y,
                                const int32_t *n_samples, int32_t max_samples_per_query,
                                float f0, uint64_t seed, uint64_t counter_base, uint32_t stream_id,
                                float *E, const int32_t *config, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* VNDF_H */
