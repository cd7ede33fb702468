/*
 * ckmpm.h -- C ABI of the GB300-native compact-kernel MPM (CK-MPM) step.
 *
 * Method: "CK-MPM: A Compact-Kernel Material Point Method" (arXiv 2412.10399).
 * One time step (Sec. 3.2 pipeline, on the dual staggered grid of Sec. 4.2):
 *   P2G   mass, APIC momentum (Sec. 4.4) and MLS stress force (Sec. 4.3.2,
 *         Sec. 4.5) scattered onto both grids G- and G+ with the compact
 *         kernel K1 (Sec. 4.1), two nodes per axis per grid;
 *   grid  m v~ = m v + dt f per grid (Sec. 4.3.3), plus gravity and sticky
 *         walls;
 *   G2P   v and B gathered from both grids (Sec. 4.3.4, Sec. 4.4), F update
 *         (Sec. 4.3.5), constitutive update (fixed-corotated, Drucker-Prager
 *         return mapping; Sec. 3.2 step 4), advection (Sec. 3.2 step 5).
 * A quadratic B-spline MLS-MPM path (single grid, 27 nodes) is built the same
 * way for comparison (Sec. 5.2 / Sec. 6.2 comparison path).  The transfer is
 * selectable per context (ckmpm_transfer): APIC + MLS as above (default), PIC
 * with the kernel gradient (Sec. 4.3), or APIC with the kernel gradient
 * (Sec. 4.4 with the force and velocity gradient of Sec. 4.3).
 *
 * Conventions
 *  - Node i of grid k in {-1 (G-), +1 (G+)} sits at (i - k/4) dx; node indices
 *    run 0..res on every axis.  Quadratic nodes sit at i dx.
 *  - Every call is made from one host thread per context; contexts are
 *    independent.  No exception crosses this ABI and no kernel traps: device
 *    errors set a status word that ckmpm_sync() reports.
 *  - Pointers marked "host or device" are interpreted per the accompanying
 *    is_device flag; device pointers must be on the context's device.
 *  - Input arrays are borrowed and copied into the context's own state; the
 *    context owns all device state.  Output arrays are owned by the caller.
 *    Calls that synchronise (ckmpm_upload, ckmpm_readback) are done with
 *    their arrays on return.  ckmpm_create and ckmpm_admit read device
 *    arrays and page-locked host arrays in stream order: those must stay
 *    unchanged until the context's stream has passed the call (the next
 *    ckmpm_sync or synchronising call); pageable host arrays are copied
 *    before the call returns.
 *  - All floating-point state is float32; parameters are given in double and
 *    rounded once.
 */
#ifndef CKMPM_H
#define CKMPM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define CKMPM_API __attribute__((visibility("default")))
#else
#define CKMPM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CKMPM_OK = 0,
  CKMPM_EINVAL = 1,     /* invalid argument or state (message in ckmpm_last_error) */
  CKMPM_ENOMEM = 2,     /* capacity or device memory exhausted (nothing changed) */
  CKMPM_ECUDA = 3,      /* a CUDA runtime call failed */
  CKMPM_EDOMAIN = 4,    /* a particle left the valid interior [0.5 dx, (res-0.5) dx) */
  CKMPM_ENONFINITE = 5, /* a non-finite particle state was produced */
  CKMPM_ETIMEOUT = 6,   /* a bounded device wait gave up */
  CKMPM_EBUSY = 7,      /* operation not allowed now (e.g. during stream capture) */
  CKMPM_ENOTFOUND = 8   /* unknown scene id */
} ckmpm_status;

typedef enum { CKMPM_KERNEL_CK = 0, CKMPM_KERNEL_QUADRATIC = 1 } ckmpm_kernel;

/* Transfer scheme, OR-ed into a kernel argument (ckmpm_create, ckmpm_config;
 * ckmpm_p2g_grids_static takes APIC_MLS and PIC); fixed for a context.
 *   CKMPM_TRANSFER_APIC_MLS (0, the default): APIC momentum with the MLS
 *     force, state B (Sec. 4.4, 4.5).
 *   CKMPM_TRANSFER_PIC: the PIC scheme of Sec. 4.3 with the kernel gradient
 *     grad w_ip = d w_ip / d x_p: P2G adds w m v - dt V0 tau grad w to node
 *     momentum; G2P gives v_p = 1/2 sum_k sum_i w v~_i and
 *     grad v_p = 1/2 sum_k sum_i v~_i (grad w_ip)^T for F <- (I + dt grad v) F.
 *     The state keeps no B: readback of B and C gives zeros and uploading B
 *     is EINVAL.
 *   CKMPM_TRANSFER_APIC_GRAD: APIC with the kernel gradient (Sec. 4.4 taken
 *     literally, "the rest as in the PIC scheme"): P2G adds
 *     w m (v + B D^-1 (x_i - x_p)) - dt V0 tau grad w; G2P gives v and B as for
 *     APIC and grad v as for PIC.  The state keeps B and the stress term
 *     separately (36 more bytes per particle per pool buffer). */
typedef enum {
  CKMPM_TRANSFER_APIC_MLS = 0,
  CKMPM_TRANSFER_PIC = 2,
  CKMPM_TRANSFER_APIC_GRAD = 4
} ckmpm_transfer;
/* Step structure, OR-ed into a kernel argument (ckmpm_create, ckmpm_config):
 *   CKMPM_STEP_G2P2G: the fused step of Sec. 5.1 (G2P of step n and P2G of
 *     step n + 1 in one kernel, after Wang 2020) in place of separate P2G and
 *     G2P kernels; APIC + MLS transfer only (else EINVAL).  Each CTA gathers
 *     a particle block of step n and scatters the particles that stay in
 *     that block into the next step's grid; particles that move to another
 *     block (or take the float64 pass) are scattered by a second, small
 *     kernel.  Results match the split step within float32 rounding.  The
 *     context keeps a second block table (one entry per virtual grid block)
 *     and a particle list.  After an admission, release, upload or probe the
 *     next step first recomputes the current grid with the split kernels. */
typedef enum { CKMPM_STEP_SPLIT = 0, CKMPM_STEP_G2P2G = 8 } ckmpm_step_mode;
typedef enum { CKMPM_FIXED_COROTATED = 0, CKMPM_DRUCKER_PRAGER = 1, CKMPM_J_FLUID = 2 } ckmpm_model;

/* Constitutive parameters of one material.  Lame parameters are
 * mu = E / (2 (1 + nu)), lambda = E nu / ((1 + nu)(1 - 2 nu)).  Drucker-Prager
 * uses Hencky elasticity and the cone alpha = sqrt(2/3) 2 sin(phi)/(3 - sin(phi))
 * with cohesion 0 (klar2016, cited in Sec. 3.2).  The J-based fluid (the
 * equation of state of the dam-break scenes in the performance section) has
 * pressure p = E (J^-gamma - 1), Kirchhoff stress -J p I, and keeps only its
 * volume ratio: F = J^(1/3) I after every update; nu and friction_deg are
 * unused for it. */
typedef struct {
  int model;            /* ckmpm_model */
  double E;             /* Young's modulus [Pa]; for the fluid the equation-of-state constant B [Pa] */
  double nu;            /* Poisson ratio */
  double rho;           /* density [kg/m^3]; particle mass = rho * dx^3 / ppc */
  double friction_deg;  /* Drucker-Prager friction angle phi [deg], in [0, 90) (else EINVAL) */
  double gamma;         /* fluid equation-of-state exponent (unused by the solids) */
} ckmpm_material;

/* One simulation ("scene"): a cubic domain [0, res*dx]^3, y up. */
typedef struct {
  int64_t n;               /* number of particles (>= 1) */
  const float* x;          /* n*3 positions, host or device; must lie in [0.5dx, (res-0.5)dx) */
  const float* v;          /* n*3 velocities or NULL (zero), host or device */
  const uint8_t* mat;      /* n material indices into materials[] or NULL (all 0) */
  int is_device;           /* 1: x, v, mat are device pointers */
  int res;                 /* cells per axis (4..4096) */
  double dx;               /* cell size; a power of two keeps x/dx exact in float32 */
  double dt;               /* time step */
  double gravity[3];       /* m/s^2 added on nodes with mass */
  double bc_cells;         /* sticky walls: v~ = 0 on nodes closer than bc_cells*dx to a wall */
  int ppc;                 /* particles per cell used to sample; particle volume V0 = dx^3/ppc */
  const ckmpm_material* materials; /* host array, copied */
  int n_materials;         /* 1..255 */
  /* Precision extension: the 3x3 SVD / polar decomposition of the constitutive
   * update is redone in float64 where |det F| < fp64_j_tol, or
   * sigma_min < fp64_cond_tol * sigma_max, or (sigma_i - sigma_j) <
   * fp64_gap_tol * sigma_max for some pair.  Zero disables a criterion. */
  double fp64_j_tol;
  double fp64_cond_tol;
  double fp64_gap_tol;
} ckmpm_scene;

/* Optional device-memory provider (for example a PyTorch caching allocator).
 * alloc returns a device pointer aligned to 256 bytes or NULL. */
typedef struct {
  void* (*alloc)(size_t bytes, void* user);
  void (*free)(void* ptr, size_t bytes, void* user);
  void* user;
} ckmpm_allocator;

/* Capacities of a multi-scene context (a "server"): all resident scenes step
 * together in one launch per kernel over their concatenated block lists.
 * Serving many scenes is an extension with no counterpart in the paper; each
 * scene's step is the method's step above, with its own dx, dt, materials,
 * gravity and walls. */
typedef struct {
  int kernel;                  /* ckmpm_kernel | ckmpm_transfer | ckmpm_step_mode; fixed for the context */
  int64_t max_particles;       /* particle pool capacity */
  int64_t max_keys;            /* particle-block key space (sum over scenes of ceil(res/4)^3) */
  int64_t max_grid_blocks;     /* grid pool: 4x4x4-node blocks active at once, all scenes together */
  int64_t max_virtual_blocks;  /* block-table entries (sum over scenes of (ceil(res/4)+1)^3) */
  int max_scenes;              /* resident scene slots (<= 1024) */
  int max_materials;           /* material table entries (<= 65535) */
  int per_particle_E;          /* 1: keep a per-particle Young's modulus (differentiation) */
  void* stream;                /* cudaStream_t to run on; NULL: the context creates one */
  const ckmpm_allocator* allocator; /* NULL: cudaMalloc / cudaFree */
} ckmpm_config;

typedef struct ckmpm_ctx ckmpm_ctx;

/* Particle and grid fields for readback / upload. */
typedef enum {
  CKMPM_FIELD_X = 0,      /* n*3 float positions (readback, upload) */
  CKMPM_FIELD_V = 1,      /* n*3 float velocities (readback, upload) */
  CKMPM_FIELD_B = 2,      /* n*9 float APIC matrix B, row-major (readback, upload; zeros and no upload under PIC) */
  CKMPM_FIELD_C = 3,      /* n*9 float affine velocity gradient C = B D(x)^-1 (readback; zeros under PIC) */
  CKMPM_FIELD_F = 4,      /* n*9 float (elastic) deformation gradient (readback, upload) */
  CKMPM_FIELD_E = 5,      /* n float per-particle Young's modulus (needs per_particle_E) */
  CKMPM_FIELD_GRID_M = 16,  /* per grid (G- then G+; one grid for quadratic) (res+1)^3 float
                               node masses of the last ckmpm_probe_grids() */
  CKMPM_FIELD_GRID_P = 17,  /* same layout, 3 floats per node: m v + dt f after P2G */
  CKMPM_FIELD_GRID_V = 18   /* same layout, 3 floats per node: v~ after the grid update */
} ckmpm_field;

typedef struct {
  int64_t n_particles;        /* particles in the pool (all scenes) */
  int64_t n_particle_blocks;  /* non-empty particle blocks in the last step */
  int64_t n_grid_blocks;      /* active grid blocks in the last step */
  int64_t steps;              /* global steps taken */
  int64_t fp64_particles;     /* particles of the last step's float64 pass */
  double ms_last_step;        /* device time of the last step (timing on) */
  double ms_kernel[8];        /* average device ms per launch per kernel since the
                                 last ckmpm_reset_timing(): 0 bin, 1 scatter,
                                 2 p2g (fused steps: the leftover P2G), 3 grid
                                 update, 4 g2p, 5 grid list, 6 float64 pass,
                                 7 fused G2P2G */
  int64_t launches_kernel[8]; /* launches counted in ms_kernel */
  int64_t launches_per_step;  /* kernel launches issued by one step */
  int64_t leftover_particles; /* fused steps: particles of the last step's leftover P2G */
  int64_t graph_steps;        /* steps launched as a CUDA graph (see ckmpm_step) */
} ckmpm_stats;

/* Create a context holding one scene (scene id 0) with capacities equal to
 * that scene.  kernel: ckmpm_kernel | ckmpm_transfer | ckmpm_step_mode.
 * stream: cudaStream_t or NULL.
 * Errors: EINVAL (bad scene), ENOMEM, ECUDA.  *out is NULL on error. */
CKMPM_API ckmpm_status ckmpm_create(const ckmpm_scene* scene, int kernel, void* stream, ckmpm_ctx** out);

/* Create an empty multi-scene context with the given capacities. */
CKMPM_API ckmpm_status ckmpm_create_server(const ckmpm_config* cfg, ckmpm_ctx** out);

/* Launch tuning read from the environment by ckmpm_create and
 * ckmpm_create_server (once, at creation; unset means the default).  They
 * change how the kernels are scheduled, never what they compute: results
 * agree to float32 rounding.
 *   CKMPM_GRAPHS=0        launch steady steps directly instead of replaying
 *                         CUDA graphs
 *   CKMPM_G2P_MINB=4|5|6  G2P register budget for the APIC + MLS transfer:
 *                         16, 20 (default) or 24 resident warps per SM
 *   CKMPM_P2G_REP=1|2     copies of the P2G shared accumulators (default: 1
 *                         for the compact kernel, 2 for the quadratic twin)
 *   CKMPM_P2G_ROT=0|1     with one copy, issue the four sums in order (0) or
 *                         in the lane-rotated order (1; compact-kernel default)
 *   CKMPM_P2G_FMA=0|1     APIC + MLS: round contributions to fixed point by a
 *                         conversion (0) or, in blocks of 256 or more
 *                         particles, by a fused multiply-add (1, default)
 *   CKMPM_SPLITS=1..8     work units per particle block (default: chosen per
 *                         step from the particle count)
 *   CKMPM_CTAS_PER_SM=k   CTAs per SM of the kernel that clears the grid
 *                         accumulators after ckmpm_probe_grids (default 8) */

/* Admit a scene into a context (continuous batching, an extension with no
 * counterpart in the paper: takes effect at the next step; resident scenes
 * keep running).  ENOMEM if any capacity would be
 * exceeded (nothing changes).  *scene_id receives the scene's id.
 * Host x, v, mat are copied into a device staging buffer on the context's
 * stream (page-locked ones asynchronously; see Conventions). */
CKMPM_API ckmpm_status ckmpm_admit(ckmpm_ctx* ctx, const ckmpm_scene* scene, int* scene_id);

/* Remove a scene; its particles leave the pool at the next step and its
 * capacity is reusable by later admissions. */
CKMPM_API ckmpm_status ckmpm_release(ckmpm_ctx* ctx, int scene_id);

/* Enqueue n time steps of every resident scene on the context's stream.
 * Each step is the pipeline of Sec. 3.2 on the dual grid of Sec. 4.2:
 * binning of the particles by particle block (Sec. 5.1), P2G onto both grids
 * (Sec. 4.3.1, 4.3.2, 4.4, 4.5), the grid update with gravity and sticky walls
 * (Sec. 4.3.3), and G2P with the F update, the constitutive update and the
 * advection (Sec. 4.3.4, 4.3.5; Sec. 3.2 steps 3-5); with CKMPM_STEP_G2P2G
 * the G2P of step k and the P2G of step k + 1 run in one kernel (Sec. 5.1).
 * Asynchronous: device-side errors (EDOMAIN, ENONFINITE) surface at the next
 * ckmpm_sync / ckmpm_readback.  Returns EINVAL for n < 0, ECUDA on a launch
 * failure, or the sticky error of an earlier step.
 * A steady step (no admission, release, upload or probe since the previous
 * one, timing off) is captured once into a CUDA graph per parity of the
 * double-buffered state and replayed after that, which saves the launch
 * gaps of its nine to eleven kernels; any of those operations drops the
 * graphs.  A stream that cannot be captured (the legacy default stream, or
 * one the caller is capturing) gets direct launches.  CKMPM_GRAPHS=0 in the
 * environment turns graphs off for contexts created afterwards. */
CKMPM_API ckmpm_status ckmpm_step(ckmpm_ctx* ctx, int n);

/* Wait for the context's stream and return the first device error (sticky). */
CKMPM_API ckmpm_status ckmpm_sync(ckmpm_ctx* ctx);

/* Run P2G (Sec. 4.3.1, 4.3.2, 4.4, 4.5) and the grid update (Sec. 4.3.3) for
 * the current state without advancing it, so that GRID_M / GRID_P / GRID_V
 * can be read back.  Enqueued on the context's stream like a step (the
 * readback of a grid field synchronises); the next step first clears the
 * probed accumulators. */
CKMPM_API ckmpm_status ckmpm_probe_grids(ckmpm_ctx* ctx);

/* Copy a field of one scene into dst (host or device), in the scene's
 * original particle order.  bytes must equal the field size exactly.  B is
 * the APIC matrix of Sec. 4.4 (the state keeps M = m B - dt V0 tau and B is
 * recovered as (M + dt V0 tau(F)) / m), C = B D(x)^-1 with D of Sec. 4.4 at
 * the particle's position.
 * Synchronises the stream.  EINVAL on a size mismatch.  A host dst goes
 * through ckmpm_readback_async + ckmpm_readback_wait (no allocation once the
 * staging slots have grown to the field's size). */
CKMPM_API ckmpm_status ckmpm_readback(ckmpm_ctx* ctx, int scene_id, int field, void* dst, size_t bytes,
                            int dst_is_device);

/* Asynchronous host readback of the same fields (a state query between steps,
 * not part of the paper's method).  Enqueues, on the context's stream, the
 * gather of the field as the steps enqueued so far leave it into one of two
 * device staging slots owned by the context, and, on a second stream of the
 * context, the copy of that slot into host_dst; returns at once with
 * *ticket >= 0.  Steps enqueued afterwards run while the copy proceeds.
 * host_dst (bytes, exactly the field size) belongs to the caller and must
 * stay valid and unread until ckmpm_readback_wait(ctx, *ticket) returns;
 * page-locked memory (cudaHostAlloc / torch pin_memory) is needed for the
 * copy to overlap, pageable memory makes the call wait for the copy.
 * Tickets alternate between the two slots: a third call reuses the first
 * slot and makes the context's stream wait (on the device, not the host)
 * until that slot's previous copy has finished.
 * Errors: as ckmpm_readback (EINVAL, ENOTFOUND, EBUSY under capture), ENOMEM
 * when a slot cannot grow, ECUDA; *ticket is -1 on error. */
CKMPM_API ckmpm_status ckmpm_readback_async(ckmpm_ctx* ctx, int scene_id, int field, void* host_dst, size_t bytes,
                                            int64_t* ticket);

/* Wait (on the host) until the copy of a ticket has reached its host buffer,
 * then return the sticky device error as it stood when the field was
 * gathered (EDOMAIN, ENONFINITE, ...).  Waiting on an older ticket than the
 * last two waits for the newest copy of its slot.  EINVAL for a ticket this
 * context never issued. */
CKMPM_API ckmpm_status ckmpm_readback_wait(ckmpm_ctx* ctx, int64_t ticket);

/* Overwrite a particle field (X, V, B, F, E) of one scene from src (host or
 * device), in the scene's original particle order.  bytes must equal the
 * field size.  Synchronises the stream. */
CKMPM_API ckmpm_status ckmpm_upload(ckmpm_ctx* ctx, int scene_id, int field, const void* src, size_t bytes,
                          int src_is_device);

/* Number of particles of a scene, or -1. */
CKMPM_API int64_t ckmpm_scene_particles(const ckmpm_ctx* ctx, int scene_id);

/* Counters of the last step; timing adds CUDA events around every kernel
 * (on the context's stream) and is off by default. */
CKMPM_API ckmpm_status ckmpm_get_stats(ckmpm_ctx* ctx, ckmpm_stats* out);
CKMPM_API ckmpm_status ckmpm_set_timing(ckmpm_ctx* ctx, int on);
CKMPM_API ckmpm_status ckmpm_reset_timing(ckmpm_ctx* ctx);

/* Release everything owned by the context.  NULL is accepted. */
CKMPM_API ckmpm_status ckmpm_destroy(ckmpm_ctx* ctx);

/* Human-readable description of the last error of ctx (never NULL). */
CKMPM_API const char* ckmpm_last_error(const ckmpm_ctx* ctx);

/* ---------------------------------------------------------------------------
 * Differentiable stepper (extension: gradients of a rollout).
 *
 * One CK-MPM step (Sec. 4.3-4.5 with readings R4-R8) as a pure function of the
 * particle state, for the fixed-corotated model, on a dense dual grid of
 * (res+1)^3 nodes per grid, with particles kept in the caller's order; and its
 * adjoint (reverse of G2P, grid update and P2G, including the derivatives of
 * the kernel weights, of D(x) and of the polar decomposition).  All state
 * arrays are float32 device arrays owned by the caller: x, v n*3; B, F n*9
 * (row-major 3x3); E n (per-particle Young's modulus).  Work is enqueued on the
 * stream given at creation; ckmpm_diff_sync waits and reports EDOMAIN if a
 * particle touched nodes outside 0..res.
 * ------------------------------------------------------------------------- */
typedef struct ckmpm_diff ckmpm_diff;

/* scene: n, res, dx, dt, gravity, bc_cells, ppc and materials[0] (must be
 * fixed-corotated; its rho and nu are used, E comes per particle).  Device
 * buffers for the dense grids are allocated here.  EINVAL / ENOMEM. */
CKMPM_API ckmpm_status ckmpm_diff_create(const ckmpm_scene* scene, void* stream, ckmpm_diff** out);

/* (x, v, B, F; E) -> (x1, v1, B1, F1); outputs must not alias inputs. */
CKMPM_API ckmpm_status ckmpm_diff_step(ckmpm_diff* d, const float* x, const float* v, const float* B,
                                       const float* F, const float* E, float* x1, float* v1, float* B1, float* F1);

/* Vector-Jacobian product of one step at (x, v, B, F; E): given the adjoints
 * (gx1, gv1, gB1, gF1) of the step's outputs, writes the adjoints (gx, gv,
 * gB, gF) of its inputs and ADDS d<adjoint, step>/dE to gE. */
CKMPM_API ckmpm_status ckmpm_diff_step_backward(ckmpm_diff* d, const float* x, const float* v, const float* B,
                                                const float* F, const float* E, const float* gx1, const float* gv1,
                                                const float* gB1, const float* gF1, float* gx, float* gv, float* gB,
                                                float* gF, float* gE);

CKMPM_API ckmpm_status ckmpm_diff_sync(ckmpm_diff* d);
CKMPM_API ckmpm_status ckmpm_diff_destroy(ckmpm_diff* d);

/* Allocation-free variant of the particle-to-grid transfer (no counterpart in
 * the paper; it exists for callers that may not allocate device memory when
 * they call: an application whose own fixed arena owns the device memory, a
 * real-time loop that cannot afford cudaMalloc's implicit synchronisation, or
 * a plug-in that must not grow the process's footprint after start-up).
 *
 * Computes for one scene the same grids as ckmpm_create + ckmpm_upload(F, B)
 * + ckmpm_probe_grids + ckmpm_readback(GRID_M, GRID_P): mass and momentum
 * (m v + dt f) of both CK grids (or the quadratic grid) after P2G.  It calls
 * no cudaMalloc, cudaFree or allocating library routine: all working memory is
 * one fixed 18 MiB device array inside the library, held on every GPU that
 * loads the library until the process exits.
 *   scene   is_device must be 1 (x, v, mat already on the current device);
 *           n <= 65536, res <= 64, n_materials <= 16, else CKMPM_EINVAL.
 *   kernel  ckmpm_kernel | ckmpm_transfer.
 *   B, F    device arrays of n*9 floats (row-major) or NULL (B = 0, F = I);
 *           B must be NULL with CKMPM_TRANSFER_PIC.
 *   grid_m  device output, (res+1)^3 floats per grid (G- then G+ for CK).
 *   grid_p  device output, (res+1)^3 * 3 floats per grid.
 *   stream  cudaStream_t or NULL; the call returns after the work finished.
 * Every call on a GPU shares that array (a previous call's leftovers are
 * cleared first), so calls that overlap on the same GPU race.  The first call
 * on each GPU looks up the array's address with that GPU current: make it
 * before any stream capture.  With CUDA's default lazy module loading that
 * first call is also when the 18 MiB are reserved on the GPU (with
 * CUDA_MODULE_LOADING=EAGER, when the library's device code is loaded): a
 * caller whose own arena will take the device memory should make one small
 * warm-up call per GPU before the arena does, since a first call without
 * 18 MiB free fails with ECUDA.  The call synchronises only its own stream
 * (the error word is read back on it).  Returns EDOMAIN / ENONFINITE for
 * particles outside the interior or non-finite input, EINVAL for a material
 * index at or above n_materials, ECUDA on a runtime error. */
CKMPM_API ckmpm_status ckmpm_p2g_grids_static(const ckmpm_scene* scene, int kernel, const float* B,
                                             const float* F, float* grid_m, float* grid_p, void* stream);

/* Library version string. */
CKMPM_API const char* ckmpm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CKMPM_H */
