/*
 * lbm.h -- C ABI of the GB300 lattice Boltzmann library for curved no-slip
 * walls: the fused collide-stream sweep with interpolated bounce-back or
 * direct-forcing immersed boundary, after Peng, Ayala & Wang, "A comparative
 * study of immersed boundary method and interpolated bounce-back scheme for
 * no-slip boundary treatment in the lattice Boltzmann method" (arXiv
 * 1906.05445).
 *
 * Units are lattice units throughout: dx = dt = h = 1, c_s^2 = 1/3 and the
 * reference density rho0 = 1.  Arrays exchanged with the caller are FP64 in
 * the layout [component][z][y][x] (x fastest; nz = 1 for D2Q9).  Directions
 * are numbered as follows (e_i):
 *   D2Q9 : 0 (0,0); 1 (1,0); 2 (0,1); 3 (-1,0); 4 (0,-1); 5 (1,1); 6 (-1,1);
 *          7 (-1,-1); 8 (1,-1)
 *   D3Q19: 0 rest; 1 +x; 2 -x; 3 +y; 4 -y; 5 +z; 6 -z; 7 (1,1,0);
 *          8 (-1,-1,0); 9 (1,-1,0); 10 (-1,1,0); 11 (1,0,1); 12 (-1,0,-1);
 *          13 (1,0,-1); 14 (-1,0,1); 15 (0,1,1); 16 (0,-1,-1); 17 (0,1,-1);
 *          18 (0,-1,1)
 *
 * Conventions of every entry point:
 *  - the return value is an lbm_status; on error the context is unchanged
 *    and lbm_last_error() describes the failure;
 *  - work is enqueued on the CUDA stream given to lbm_create; the calls
 *    that return data to the host (queries, lbm_sync, lbm_save) synchronise
 *    that stream and report any CUDA error raised by earlier work;
 *  - host buffers belong to the caller and are only read or written during
 *    the call; device memory belongs to the library;
 *  - a context is not thread-safe; distinct contexts may share a stream;
 *  - every simulation step runs in the library's CUDA kernels: there is no
 *    CPU path, and a missing or unusable GPU is an error (LBM_ERR_CUDA).
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
  LBM_OK = 0,
  LBM_ERR_ARG = -1,         /* invalid argument or descriptor */
  LBM_ERR_OOM = -2,         /* device or host allocation failed */
  LBM_ERR_CUDA = -3,        /* CUDA runtime error (message in last_error) */
  LBM_ERR_UNSUPPORTED = -4, /* valid but not implemented combination */
  LBM_ERR_STATE = -5,       /* call not valid in the current state */
  LBM_ERR_TIMEOUT = -6,     /* a host-side wait ran out (lbm_server_wait), or a kernel's bounded
                               wait for its own asynchronous copies gave up (lbm_sync) */
  LBM_ERR_DIVERGED = -7,    /* non-finite residual */
  LBM_ERR_CAPACITY = -8     /* a fixed-capacity device list overflowed */
} lbm_status;

/* lattice selectors */
enum { LBM_D2Q9 = 0, LBM_D3Q19 = 1 };
/* collision operators: Eq. 1 (BGK) and Eq. 3 (MRT) */
enum { LBM_BGK = 0, LBM_MRT = 1 };
/* storage / compute precision of the distributions */
enum {
  LBM_FP64 = 0,           /* FP64 storage and arithmetic (parity build) */
  LBM_FP32 = 1,           /* FP32 storage of f - w_i, FP32 arithmetic */
  LBM_FP32_BF16STORE = 2, /* BF16 storage of f - w_i, FP32 arithmetic */
  LBM_FP32_FP16STORE = 3  /* FP16 storage of scaled f - w_i, FP32 arithmetic */
};
/* Accuracy of the 16-bit storage paths.  A storage precision is accepted
 * for a flow only where its drag error against the FP64 result stays below
 * 10% of the discretisation error at that resolution (Richardson estimate
 * from twice the resolution).  Measured:
 *  - fixed sphere, R = 3.75 in a 40^3 periodic box, tau = 0.6, g = 3.4e-8
 *    (flow speed ~1e-4), 2000 steps: FP16 meets it under IBM (0.05-0.8%) but
 *    not under quadratic Bouzidi (24%); BF16 meets it under neither (IBM
 *    3-19% from run to run, Bouzidi 366%);
 *  - sphere translating at U = 0.01 (R = 8, 20000 steps): FP16 meets it
 *    under both schemes (4.8% / 0.46%); BF16 under IBM only (9.7%), not
 *    under Bouzidi with refilling (216%).
 * BF16 storage with any bounce-back scheme therefore does not meet the rule
 * in any flow measured; use FP32 or FP16 storage there.  The library does
 * not refuse the combination: it is a fast, less accurate option. */
/* where the external body force acts */
enum { LBM_FORCE_FLUID_ONLY = 0, LBM_FORCE_ALL = 1 };
/* solid shapes */
enum { LBM_SPHERE = 0, LBM_CYLINDER_Z = 1 };
/* no-slip schemes (Sec. 2.1 and Sec. 2.2 of the paper) */
enum {
  LBM_SCHEME_NONE = 0,    /* solids ignored: periodic box */
  LBM_BOUNCE_BACK = 1,    /* Eq. 10 */
  LBM_BOUZIDI_LIN = 2,    /* two-point form of Eq. 11 */
  LBM_BOUZIDI_QUAD = 3,   /* Eq. 11 */
  LBM_YU_LIN = 4,         /* two-point form of Eqs. 12-14 */
  LBM_YU_QUAD = 5,        /* Eqs. 12-14 (the combined Eq. 15) */
  LBM_IBM_DIRECT = 6,     /* direct-forcing IBM, Eqs. 4-9 */
  LBM_ZHAO_YONG = 7       /* single-node bounce-back, Eq. 16 (solids at rest or
                             rotating in place; translating solids are
                             LBM_ERR_UNSUPPORTED, and so is lbm_save; select
                             it before stepping or after an initialisation,
                             else LBM_ERR_STATE) */
};
/* fields for lbm_device_field */
enum { LBM_FIELD_F_POST = 0, LBM_FIELD_FLAGS = 1 };

/* Lattice: Eq. 1 / Eq. 3 with nu = (tau - 1/2)/3 (Eq. 2).
 * mrt_rates: relaxation rate per moment (order of the Gram-Schmidt basis:
 *   D2Q9  rho, e, eps, jx, qx, jy, qy, pxx, pxy;
 *   D3Q19 rho, e, eps, jx, qx, jy, qy, jz, qz, 3pxx, 3pixx, pww, piww, pxy,
 *         pyz, pxz, mx, my, mz);
 *   0 selects the default: 1/tau, except the energy-flux moments q whose rate
 *   satisfies (tau - 1/2)(1/s_q - 1/2) = 3/16.  The stress rates are always
 *   1/tau and the conserved moments' rates have no effect.
 * body_force: uniform force density g (acts on nodes outside every solid
 *   unless force_region == LBM_FORCE_ALL). */
typedef struct {
  int lattice;
  int nx, ny, nz;
  double tau;
  int collision;
  double mrt_rates[19];
  int precision;
  double body_force[3];
  int force_region;
} lbm_lattice_desc;

/* Solid: a sphere (a circle on D2Q9) or a cylinder along z.
 * fluid_inside = 0: the solid is the ball |x - c| <= R;
 * fluid_inside = 1: the solid is the outside |x - c| >= R (an enclosing
 *   wall, e.g. the outer cylinder of a Couette cell or a pipe).
 * velocity: translation speed; the centre moves by velocity per step.
 * omega: angular velocity; the wall velocity is u_w = U + omega x (x_w - c).
 * Distances use the nearest periodic image. */
typedef struct {
  int kind;
  double centre[3];
  double radius;
  double velocity[3];
  double omega[3];
  int fluid_inside;
} lbm_solid_desc;

/* delta-function kernels of the IBM (Sec. 3.1 compares the first three) */
enum {
  LBM_DELTA_PESKIN4 = 0, /* Peskin's 4-point kernel, Eq. 6 (default) */
  LBM_DELTA_ROMA3 = 1,   /* Roma, Peskin & Berger's 3-point kernel */
  LBM_DELTA_LINEAR2 = 2, /* 2-point linear kernel */
  LBM_DELTA_COSINE4 = 3  /* 4-point cosine kernel (Appendix B) */
};

/* inertia of the fluid inside a free solid under IBM (Sec. 3.2) */
enum {
  LBM_INERTIA_FENG = 0, /* rigid-body inside fluid, Feng & Michaelides, Eq. 23 (default) */
  LBM_INERTIA_KEMPE = 1, /* Kempe et al.: volume integrals over level-set cell fractions,
                            Eqs. 24-26 */
  LBM_INERTIA_UHLMANN = 2 /* Uhlmann: the inside fluid's inertia taken off the solid's,
                             Eq. 22; needs rho_p > rho_f (LBM_ERR_ARG otherwise) and is
                             unstable below a density ratio of about 2 in 2D */
};

/* Scheme.  For LBM_IBM_DIRECT: ibm_iters >= 1 forcing iterations (Eq. 9
 * applied to the spread force), ibm_retraction = R_d (markers at R - R_d, or
 * R + R_d for an enclosing wall), ibm_marker_density = markers per unit
 * surface area (per unit length in 2D), 0 -> 1, ibm_kernel = LBM_DELTA_*
 * (zero-initialised descriptors get Peskin's kernel), ibm_inertia =
 * LBM_INERTIA_* for free solids (lbm_set_solid_dynamics).  An unknown kernel
 * or inertia treatment is LBM_ERR_ARG. */
typedef struct {
  int scheme;
  int ibm_iters;
  double ibm_retraction;
  double ibm_marker_density;
  int ibm_kernel;
  int ibm_inertia;
} lbm_scheme_desc;

typedef struct {
  int64_t nodes;          /* nx * ny * nz */
  int64_t fluid_nodes;    /* nodes carrying distributions */
  int64_t list_nodes;     /* nodes handled by the boundary-node kernel */
  int64_t cut_links;      /* interpolated bounce-back links */
  int64_t markers;        /* IBM markers over all solids */
  int64_t steps;          /* steps taken since create */
  int64_t kernel_launches;/* kernels launched since create */
  int64_t device_bytes;   /* device memory held */
  int32_t num_solids;
  int32_t precision;
  int32_t bulk_kernel;    /* bulk sweep of the last single-lattice step: 0 one node
                             per thread, 1 vectors of nodes per thread, 2 vectors fed
                             by bulk copies of row segments; -1 before the first */
} lbm_info;

/* Create a lattice at rest (f = w_i, no solids, scheme NONE) on the current
 * CUDA device.  cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * Errors: LBM_ERR_ARG (bad sizes/tau/selectors), LBM_ERR_OOM, LBM_ERR_CUDA. */
lbm_status lbm_create(lbm_ctx **out, const lbm_lattice_desc *desc,
                      void *cuda_stream);
void lbm_destroy(lbm_ctx *ctx);

/* Add a solid (at most 8).  Geometry (Fig. 1: solid nodes, cut links, wall
 * fractions q) is rebuilt before the next step. */
lbm_status lbm_add_solid(lbm_ctx *ctx, const lbm_solid_desc *solid,
                         int *solid_id);
/* Replace the centre, velocity and angular velocity of a solid. */
lbm_status lbm_set_solid_motion(lbm_ctx *ctx, int solid_id,
                                const double centre[3],
                                const double velocity[3],
                                const double omega[3]);
lbm_status lbm_set_scheme(lbm_ctx *ctx, const lbm_scheme_desc *scheme);

/* Domain faces (Sec. 3.4, the uniform flow past a sphere in an open box).
 * type[k] for the faces x-, x+, y-, y+, z-, z+; u[k] the velocity of a
 * LBM_FACE_VELOCITY face.  A non-periodic face lies half a spacing outside
 * the outermost nodes:
 *  - LBM_FACE_VELOCITY: a plane wall moving with u[k] (a velocity inlet, or a
 *    no-slip wall with u = 0): the populations leaving the domain bounce back
 *    with the moving-wall term, f_i = f*_ib + 2 rho0 w_i e_i.u / cs^2;
 *  - LBM_FACE_FREE_SLIP: stress-free (no normal velocity, no shear stress):
 *    specular reflection;
 *  - LBM_FACE_CONVECTIVE: outflow, d(rho0 u)/dt + U_o d(rho0 u)/dn = 0 on each
 *    unknown population, upwind and implicit in the inner neighbour, U_o the
 *    outward velocity at the face node in the previous step (clamped at 0).
 * A link crossing two faces takes a velocity face's rule first, then the
 * outflow's, then free slip.  The default is periodic on every face.
 * Errors: LBM_ERR_ARG for an unknown type, a periodic face whose opposite
 * face is not, a z face on a 2D lattice, a second outflow face or a
 * non-periodic axis shorter than 3 nodes; LBM_ERR_STATE for an outflow face
 * set after stepping (set it first, or right after lbm_init_equilibrium /
 * lbm_set_distributions).  A solid's surface must keep 1.5 spacings clear
 * of the outermost nodes at a velocity or stress-free face (interpolation
 * nodes of the bounce-back rules beyond the face count as missing) and
 * R + 5 nodes at an outflow face, and solids may be neither fluid-inside
 * nor z-cylinders crossing non-periodic z faces: else the next step or
 * query returns LBM_ERR_UNSUPPORTED.  Checkpoints of a lattice with an outflow face are
 * LBM_ERR_UNSUPPORTED.  NULL restores the periodic box. */
enum {
  LBM_FACE_PERIODIC = 0,
  LBM_FACE_VELOCITY = 1,
  LBM_FACE_FREE_SLIP = 2,
  LBM_FACE_CONVECTIVE = 3
};
typedef struct {
  int type[6];
  double u[6][3];
} lbm_domain_desc;
lbm_status lbm_set_domain(lbm_ctx *ctx, const lbm_domain_desc *domain);

/* Set the state to the equilibrium at (rho, u) on every fluid node. */
lbm_status lbm_init_equilibrium(lbm_ctx *ctx, double rho, const double u[3]);
/* Set / read the pre-collision distributions f(x, t) (full f, not f - w):
 * host array of n = Q * nodes doubles, [Q][z][y][x].  Values at solid nodes
 * are ignored on input and returned as 0.  The upload needs no device
 * allocation: it is copied in chunks of up to 2^20 doubles through staging
 * space inside the distribution array that the next step overwrites, and
 * converted on the device to the storage type while the next chunk is
 * copied.  lbm_set_distributions returns when the upload is complete. */
lbm_status lbm_set_distributions(lbm_ctx *ctx, const double *host_f, size_t n);
/* The same upload without waiting: it is ordered on the context's stream
 * (later steps and queries see it).  host_f must stay valid and unchanged
 * until a synchronising call (lbm_sync, a query) returns; page-locked memory
 * (e.g. cudaHostAlloc) makes the copies asynchronous.  CUDA errors are
 * reported by the next synchronising call. */
lbm_status lbm_set_distributions_async(lbm_ctx *ctx, const double *host_f, size_t n);
lbm_status lbm_get_distributions(lbm_ctx *ctx, double *host_f, size_t n);

/* Advance nsteps time steps (asynchronous).  One step: geometry of moving
 * solids and refilling of uncovered nodes, IBM forcing (Sec. 2.1), the fused
 * pull collide-stream sweep with interpolated bounce-back on cut links
 * (Sec. 2.2) and the momentum exchange of Eq. 17. */
lbm_status lbm_step(lbm_ctx *ctx, int nsteps);
/* Advance n distinct lattices nsteps steps together (asynchronous): each
 * step runs every lattice's boundary and IBM work as lbm_step does, and the
 * bulk sweeps of lattices with the same lattice, collision and storage as
 * one grouped launch (up to 8 lattices per launch) on the first one's stream;
 * lattices on other streams are joined to it with events.  Results equal
 * those of lbm_step on each lattice.  The grouped launch's kernel time is
 * recorded on its first lattice (lbm_get_kernel_time, LBM_TIME_BULK), with
 * the bulk nodes of the whole group.  LBM_ERR_ARG for a NULL or repeated
 * lattice; any lattice's error stops the call (its message is on it). */
lbm_status lbm_step_multi(lbm_ctx *const *ctxs, int n, int nsteps);
/* Step in blocks of check_every until the velocity residual
 * ||u^n - u^(n-K)||_2 / ||u^n||_2 over fluid nodes drops below tol or
 * max_steps is reached.  LBM_ERR_DIVERGED on a non-finite residual. */
lbm_status lbm_run_to_steady(lbm_ctx *ctx, double tol, int check_every,
                             int max_steps, int *steps_done, double *residual);

/* Fields at the current time (synchronous), 0 at solid nodes:
 * density [nodes]; velocity [d][nodes] with the half-force correction;
 * strain rate [d(d+1)/2][nodes] from non-equilibrium moments (Sec. 3.1,
 *   Eq. 19 generalised), order xx, yy, xy (2D) / xx, yy, zz, xy, yz, xz (3D);
 * stress = -c_s^2 rho I + 2 rho0 nu S, same order;
 * dissipation rate epsilon = 2 nu s_ij s_ij (Sec. 3.1) [nodes]. */
lbm_status lbm_get_density(lbm_ctx *ctx, double *host_out, size_t n);
lbm_status lbm_get_velocity(lbm_ctx *ctx, double *host_out, size_t n);
/* The velocity field of lbm_get_velocity, copied to host_out without
 * waiting: the query and its copy are enqueued on the context's stream after
 * the work already there, and the call returns; lbm_sync waits for them.
 * host_out (d * nodes doubles, as lbm_get_velocity) must stay valid and
 * unread until then, and should be page-locked (e.g. cudaHostAlloc) for the
 * copy to be asynchronous.  Later steps and queries of the context are
 * ordered after the copy, so queries of several contexts on their own
 * streams overlap.  The first query of a context allocates its staging
 * buffer (and waits for the stream); errors as lbm_get_velocity. */
lbm_status lbm_get_velocity_async(lbm_ctx *ctx, double *host_out, size_t n);
lbm_status lbm_get_strain_rate(lbm_ctx *ctx, double *host_out, size_t n);
lbm_status lbm_get_stress(lbm_ctx *ctx, double *host_out, size_t n);
lbm_status lbm_get_dissipation(lbm_ctx *ctx, double *host_out, size_t n);
/* 1 where the node carries no distributions (solid under bounce-back). */
lbm_status lbm_get_solid_mask(lbm_ctx *ctx, unsigned char *host_out, size_t n);

/* Force and torque on a solid (FP64): under bounce-back the momentum
 * exchange of Eq. 17 during the most recent streaming; under IBM minus the
 * sum of marker forces times their control volume at the current time. */
lbm_status lbm_get_force_torque(lbm_ctx *ctx, int solid_id, double F[3],
                                double T[3]);
/* Free motion of a solid (Sec. 3.2): density_ratio = rho_p / rho_f > 0
 * makes the solid free, <= 0 returns it to prescribed motion; gravity acts
 * on it (the fluid feels only the lattice body force).  Every step then sets
 * its velocities from its hydrodynamic force and torque: Eq. 20 under
 * bounce-back, under IBM the Feng & Michaelides discretisation of Eq. 23
 * or, with ibm_inertia = LBM_INERTIA_KEMPE, rho_f times the change over the
 * last step of the inside fluid's momentum and angular momentum summed with
 * the level-set cell fractions of Eqs. 24-26, or with LBM_INERTIA_UHLMANN
 * Eq. 22 (dt = 1, rho_f = 1); its
 * centre moves by the mean of the old and new
 * velocity.  Spheres have V = 4/3 pi R^3 and I = 2/5 m R^2; cylinders
 * V = pi R^2 (times nz in 3D) and I = 1/2 m R^2 about z, turning about z
 * only.  LBM_ERR_STATE without a bounce-back or IBM scheme;
 * LBM_ERR_UNSUPPORTED under LBM_ZHAO_YONG.  The solids' state then lives in
 * device memory and a one-thread-per-solid kernel advances it at the end of
 * every step, on the context's stream, with no read-back; the solid queries
 * (velocity, centre, force) wait for that stream.  A solid that comes closer
 * to a non-periodic face than lbm_set_domain allows is reported by the next
 * lbm_sync as LBM_ERR_UNSUPPORTED. */
lbm_status lbm_set_solid_dynamics(lbm_ctx *ctx, int solid_id, double density_ratio,
                                  const double gravity[3]);
/* The solid's current velocity and angular velocity. */
lbm_status lbm_get_solid_velocity(lbm_ctx *ctx, int solid_id, double U[3], double Om[3]);
/* The same record (Fx Fy Fz Tx Ty Tz) copied to host_out without waiting:
 * the copy runs on a copy stream of the context, after the work already
 * enqueued on the context's stream, and later steps do not wait for it.  A
 * caller that reads the force every step keeps the GPU busy and waits once
 * with lbm_sync (which also waits for the copies) before reading the values.
 * host_out must stay valid until then, and should be page-locked (e.g.
 * cudaHostAlloc) for the copy to be asynchronous.  CUDA errors are reported
 * by the next synchronising call. */
lbm_status lbm_copy_force_torque_async(lbm_ctx *ctx, int solid_id, double *host_out);
/* The last min(max_steps, steps kept) records, oldest first, 6 doubles
 * (Fx Fy Fz Tx Ty Tz) per step; *n receives the count. */
lbm_status lbm_get_force_history(lbm_ctx *ctx, int solid_id, double *host_out,
                                 size_t max_steps, size_t *n);
lbm_status lbm_get_residual(lbm_ctx *ctx, double *residual);
lbm_status lbm_get_solid_centre(lbm_ctx *ctx, int solid_id, double centre[3]);
lbm_status lbm_get_info(lbm_ctx *ctx, lbm_info *info);

/* Borrowed device pointer to an internal field, valid until the next call
 * that steps or rebuilds the context.  LBM_FIELD_F_POST: the post-collision
 * deviations f* - w_i in the storage type, [Q][z][y][x] with *dir_stride
 * elements between consecutive directions (>= nodes: the arrays are padded);
 * LBM_FIELD_FLAGS: one byte per node.  bytes / dir_stride may be NULL. */
lbm_status lbm_device_field(lbm_ctx *ctx, int which, void **dptr,
                            size_t *bytes, size_t *dir_stride);

/* Checkpoint: the full state (distributions, flags of the current geometry,
 * solids with their motion and free-body state, scheme, step count) into a
 * caller-owned host buffer.  With host_buf == NULL *size receives the size.
 * The lattice description and the domain faces are not in it: lbm_load
 * takes a context created with the same lattice (LBM_ERR_ARG otherwise) and
 * keeps that context's faces.  LBM_ERR_UNSUPPORTED under LBM_ZHAO_YONG or
 * with an outflow face (their kept boundary state is not saved). */
lbm_status lbm_save(lbm_ctx *ctx, void *host_buf, size_t *size);
lbm_status lbm_load(lbm_ctx *ctx, const void *host_buf, size_t size);

/* Per-kernel device timing with CUDA events on the stream each kernel runs
 * on.  kernel: 0 bulk sweep, 1 boundary-node sweep, 2 IBM (all kernels),
 * 3 geometry.  enable: 0 off, 1 every kind, otherwise a mask with bit
 * (kernel + 1) set for each kind to time.  every >= 1: only the launches of
 * steps whose index is a multiple of `every` are timed.  Each timed launch
 * adds two event records to its stream, which cost the step a few
 * microseconds, so timing only the bulk sweep (enable = 2) on a sample of
 * steps disturbs the step least.  Totals since the last reset, in ms, with
 * launch counts and the number of node updates done by the timed launches. */
lbm_status lbm_set_timing(lbm_ctx *ctx, int enable, int every);
lbm_status lbm_get_kernel_time(lbm_ctx *ctx, int kernel, double *total_ms,
                               int64_t *launches, int64_t *node_updates);

/* Velocity query that allocates no device memory.  The paper has no
 * counterpart: this is an operational variant of lbm_get_velocity for
 * callers that must not allocate GPU memory once they are set up -- for
 * example a host application that has handed the remaining device memory to
 * its own pool allocator, or a time-critical loop where a cudaMalloc would
 * synchronise the device.  lbm_get_velocity allocates its FP64 staging
 * buffer the first time it is called; this variant stages the field through
 * a fixed array compiled into the library instead: 2^20 doubles (8 MiB).
 * The array is committed on a GPU by the first lbm_create on it (which also
 * looks up its device address, with that device current) and is held until
 * the process exits; the query itself then needs no set-up.
 *  - Output: as lbm_get_velocity, [d][z][y][x] FP64 into host_out (n >= d *
 *    nodes); 0 at solid nodes.
 *  - d * nodes above 2^20 is rejected with LBM_ERR_CAPACITY.
 *  - The context must not hold a pending geometry change (rebuilding it
 *    would allocate): call lbm_step or lbm_sync after add_solid / set_scheme
 *    / set_solid_motion, otherwise LBM_ERR_STATE.  The context's device must
 *    be current (LBM_ERR_STATE otherwise).
 *  - All calls, from every context, share the one array and it keeps the
 *    previous call's contents (the call clears the part it uses).  Calls
 *    whose work overlaps on the GPU (contexts on different streams, or
 *    several host threads) race on it: serialise them.
 *  - Synchronous, like the other queries. */
lbm_status lbm_get_velocity_noalloc(lbm_ctx *ctx, double *host_out, size_t n);

lbm_status lbm_sync(lbm_ctx *ctx);
const char *lbm_last_error(const lbm_ctx *ctx);

/* ---- batches: many lattices of uneven size advanced together ----
 * (workload shaped like a grid-convergence sweep: one solve per resolution).
 * lbm_batch_create takes n distinct, configured and initialised contexts
 * on one device.  It prepares them (geometry, initial collision), gives
 * each a private stream and, when autotune_blocks != 0, picks the bulk and
 * boundary-node block widths per lattice shape by timing the kernels into a
 * scratch buffer (the simulation state is untouched).  While in a batch the
 * contexts must be stepped only through the batch; their queries remain
 * valid, and a context reconfigured between batch calls (scheme, solids,
 * domain, populations) steps from its new configuration: every such call
 * makes the captured graph stale, and the next batch call prepares the
 * context and captures again.  lbm_batch_destroy gives the contexts their streams back (it does
 * not destroy them).  The batch runs on private streams but is ordered on
 * cuda_stream: lbm_batch_step and lbm_batch_run_to_steady start after the
 * work already queued there, and work queued there afterwards (an event, a
 * copy) waits for them; the contexts' queries wait for them as well.
 * Stepping captures one step pair of every lattice with static solids into
 * a CUDA graph whose per-lattice chains are independent branches, and
 * replays it: two steps of the whole batch per launch.  Lattices with
 * moving solids step directly.  Under graph replay the force history keeps
 * only the last two records per lattice (lbm_get_force_torque is exact).
 * lbm_batch_run_to_steady runs every lattice to its own residual < tol
 * (checked every check_every steps, as lbm_run_to_steady), drops converged
 * lattices from the graph, and reports steps_done[i] and residual[i]. */
typedef struct lbm_batch lbm_batch;
lbm_status lbm_batch_create(lbm_batch **out, lbm_ctx *const *ctxs, int n,
                            void *cuda_stream, int autotune_blocks);
void lbm_batch_destroy(lbm_batch *batch);
lbm_status lbm_batch_step(lbm_batch *batch, int nsteps);
lbm_status lbm_batch_run_to_steady(lbm_batch *batch, double tol,
                                   int check_every, int max_steps,
                                   int64_t *steps_done, double *residual);
/* block widths chosen for lattice i and the number of graph launches */
lbm_status lbm_batch_info(lbm_batch *batch, int i, int *bulk_block,
                          int *list_block, int64_t *graph_launches);
const char *lbm_batch_last_error(const lbm_batch *batch);
/* ---- serving: a stream of solves under continuous batching ----
 * A server owns a worker thread on the device that was current at
 * lbm_server_create.  lbm_server_submit queues a solve (a lattice, its
 * solids and scheme, an initial equilibrium state); the worker admits
 * queued solves in submission order while the device memory of the running
 * lattices plus the next one's estimate (two distribution arrays, flags and
 * solid ids, the IBM fields, the two FP64 velocity snapshots of the residual
 * and, with keep_velocity, the FP64 staging of the final velocity query)
 * stays within hbm_budget bytes (a solve that exceeds it alone runs by
 * itself).  A running lattice is counted at its memory after creation plus
 * the buffers it allocates later (the snapshots and the staging).  The
 * worker steps the running lattices together as an lbm_batch in rounds of
 * check_every steps and retires each lattice when its velocity residual
 * falls below tol (lbm_run_to_steady's measure: DONE), after max_steps steps
 * without that (UNCONVERGED, with the results at max_steps), or on a
 * non-finite residual (FAILED with LBM_ERR_DIVERGED; the other lattices of
 * the round go on unaffected).  Solves that arrive while others run join at
 * the next round.  The contexts, streams and memory are the server's; the
 * caller sees only request ids and results.
 * lbm_server_submit: LBM_ERR_ARG for a bad request (checked as lbm_create,
 * lbm_add_solid and lbm_set_scheme would); LBM_ERR_STATE after shutdown.
 * lbm_server_poll: the result so far (status PENDING, RUNNING, DONE,
 * UNCONVERGED or FAILED, with the lbm_status of the failure in error);
 * LBM_ERR_ARG for an unknown id.  lbm_server_wait: waits up to timeout_s
 * seconds (< 0: without limit) for DONE, UNCONVERGED, FAILED or CANCELLED;
 * LBM_ERR_TIMEOUT when the time runs out.
 * lbm_server_velocity: the final velocity field [d][nodes] of a DONE or
 * UNCONVERGED request submitted with keep_velocity; LBM_ERR_STATE otherwise.  A request
 * with a deadline that is still queued or running when it passes fails with
 * error LBM_ERR_TIMEOUT (checked at admission and at each round's end).
 * lbm_server_destroy finishes the running round, drops queued solves and
 * joins the worker.  Times are seconds since lbm_server_create. */
enum {
  LBM_REQ_PENDING = 0,
  LBM_REQ_RUNNING = 1,
  LBM_REQ_DONE = 2,
  LBM_REQ_FAILED = 3,   /* error: the lbm_status (LBM_ERR_TIMEOUT past the deadline,
                           LBM_ERR_DIVERGED on a non-finite residual) */
  LBM_REQ_CANCELLED = 4,
  LBM_REQ_UNCONVERGED = 5 /* max_steps reached with the residual still >= tol */
};
typedef struct {
  lbm_lattice_desc lattice;
  int nsolids; /* 0..8 */
  lbm_solid_desc solids[8];
  lbm_scheme_desc scheme;
  double rho0, u0[3]; /* initial equilibrium (rho0 <= 0: 1) */
  int keep_velocity;  /* keep the final velocity field for lbm_server_velocity */
  double deadline_s;  /* > 0: seconds after submission by which the solve must be done */
} lbm_request;
typedef struct {
  int status;
  int error;
  int64_t steps;
  double residual;
  double force[3], torque[3]; /* solid 0, zero without solids */
  double submit_s, start_s, finish_s;
  int64_t device_bytes;       /* device memory counted for the lattice while it ran (or,
                                 if larger, what it held at the end) */
} lbm_result;
typedef struct lbm_server lbm_server;
lbm_status lbm_server_create(lbm_server **out, size_t hbm_budget, double tol, int check_every,
                             int max_steps);
lbm_status lbm_server_submit(lbm_server *server, const lbm_request *request, int64_t *id);
lbm_status lbm_server_poll(lbm_server *server, int64_t id, lbm_result *result);
lbm_status lbm_server_wait(lbm_server *server, int64_t id, lbm_result *result, double timeout_s);
lbm_status lbm_server_velocity(lbm_server *server, int64_t id, double *host_out, size_t n);
/* Cancels a request: a queued one at once, a running one at the end of the
 * current round (its lattice is freed then).  LBM_ERR_ARG for an unknown id;
 * LBM_ERR_STATE if it has already finished. */
lbm_status lbm_server_cancel(lbm_server *server, int64_t id);
void lbm_server_destroy(lbm_server *server);

/* Fault injection for tests: after n more device allocations (any context,
 * any thread) every allocation fails with LBM_ERR_OOM until the hook is reset
 * with n < 0.  The failing call leaves its context usable or destroyed as
 * its own error contract states; no device memory is touched. */
void lbm_debug_fail_allocations_after(long long n);

/* Library version string. */
const char *lbm_version(void);

#ifdef __cplusplus
}
#endif
#endif
