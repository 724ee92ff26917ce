/*
 * tgv.h -- C-ABI of the B300 (sm_103a) histogram + TGV primal-dual library.
 *
 * The calls follow the problem statement of "Out-of-Core Surface Reconstruction
 * via Global TGV Minimization" (arXiv 2107.14790): aligned depth maps
 * (Sec. 3.1) are turned into per-voxel visibility histograms (Sec. 3.4, Alg. 1,
 * Sec. 4.4), the TGV functional of Eq. 2-3 is minimised by primal-dual
 * iterations (Sec. 3.2, Sec. 4.5), and the indicator field u, whose zero level
 * set is the surface, is read back (Sec. 4.6).
 *
 * Conventions shared by every call
 *  - Domain: a level is a set of 8x8x8-voxel bricks given by integer brick
 *    coordinates (Sec. 3.3 bounds the neighbours per cube; here every brick has
 *    a fixed neighbour table).  Voxel (i,j,k) of brick (bx,by,bz) is the global
 *    voxel (8bx+i, 8by+j, 8bz+k) with centre origin + (index + 0.5) * h.
 *    Voxel order in every host/device array exchanged through this ABI: active
 *    brick b in the order given at creation, then local index i + 8j + 64k.
 *    Multi-component fields are voxel-major: element [voxel * ncomp + c].
 *  - Frozen bricks (Sec. 4.5, set B): bricks outside the solved set whose u and
 *    v are constants.  A voxel link into a frozen brick uses those constants;
 *    a link to a position in neither set is "none" (no difference is taken).
 *  - Ownership: the domain owns all of its device state.  The caller owns every
 *    input and output buffer; a device input must stay valid until the
 *    domain's stream has reached the call.  Pointers may be host or device
 *    memory wherever a call says "host or device" (detected per call).
 *  - Streams: all device work of a domain runs on the CUDA stream given at
 *    creation (NULL = legacy default stream).  Calls that return host data
 *    synchronise that stream.
 *  - Errors: every call returns a tgv_status and never throws across the ABI.
 *    A CUDA error is sticky: later calls on that domain return TGV_ERR_STATE.
 *    tgv_last_error() gives a message for the last failure on a domain.
 *  - Device code requires sm_103a (B300).
 */
#ifndef TGV_H_
#define TGV_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define TGV_API __attribute__((visibility("default")))
#else
#define TGV_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TGV_OK = 0,
    TGV_ERR_INVALID_ARG = 1,   /* bad pointer, size, index or parameter */
    TGV_ERR_OUT_OF_MEMORY = 2, /* device or host allocation failed */
    TGV_ERR_BUDGET = 3,        /* a stated limit would be exceeded (vote counts, HBM budget) */
    TGV_ERR_CUDA = 4,          /* a CUDA runtime call failed */
    TGV_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up (the domain becomes unusable) */
    TGV_ERR_STATE = 6,         /* the domain is unusable after an earlier CUDA error */
    TGV_ERR_UNSUPPORTED = 7    /* a recognised option that is not built */
} tgv_status;

/* Storage type of v, vbar, p, q (u and ubar are always FP32; arithmetic is FP32).
 * FX16: v and vbar in FP16; p and q as 16-bit fixed point scaled by the radius of the
 * ball their projection keeps them in (Eq. 2's constraints |p| <= alpha1, |q|_F <=
 * alpha0): the stored integer is round(x * 32767 / alpha), so the step is alpha / 32767
 * everywhere in the ball instead of FP16's 2^-11 relative step near its edge.  Same
 * bytes as FP16; not a form of the paper (which keeps everything in floating point). */
enum { TGV_STORAGE_FP32 = 0, TGV_STORAGE_BF16 = 1, TGV_STORAGE_FP16 = 2, TGV_STORAGE_FX16 = 3 };

/* Histogram bin centres c_b (the data term sum_b h_b |u - c_b|, Sec. 3.4).
 * ENDPOINTS: c_b = -1 + 2b/(n-1)  (bin 0 = occluded -1, bin n-1 = free space +1)
 * MIDPOINTS: c_b = -1 + (2b+1)/n */
enum { TGV_CENTRES_ENDPOINTS = 0, TGV_CENTRES_MIDPOINTS = 1 };

/* Field ids for tgv_extract_field / tgv_set_field, with their component counts. */
enum {
    TGV_FIELD_U = 0,    /* 1 component */
    TGV_FIELD_UBAR = 1, /* 1 */
    TGV_FIELD_V = 2,    /* 3: v_x, v_y, v_z */
    TGV_FIELD_VBAR = 3, /* 3 */
    TGV_FIELD_P = 4,    /* 3 */
    TGV_FIELD_Q = 5     /* 6: q_xx, q_yy, q_zz, q_xy, q_xz, q_yz (symmetric) */
};

enum { TGV_PINHOLE = 0, TGV_SPHERICAL = 1 };

/* Form of the fused iteration kernel (same arithmetic):
 * PAIRED:    persistent CTAs stream each brick's state into shared memory with
 *            bulk asynchronous copies (two bricks in flight per CTA); each
 *            thread owns an x-adjacent voxel pair (default);
 * PIPELINED: the same pipeline with one voxel per thread;
 * ONE_BRICK_PER_CTA: one CTA per brick, plain loads.
 */
enum { TGV_ITER_PIPELINED = 0, TGV_ITER_ONE_BRICK_PER_CTA = 1, TGV_ITER_PAIRED = 2 };

/* Form of the histogram kernel of tgv_accumulate_depthmap(s) (identical counts):
 * GATHER:  one thread per voxel evaluates Alg. 1 for every map of a launch and
 *          adds its votes to its own words once (default);
 * SCATTER: one thread per depth-pyramid pixel walks the voxels its frustum can
 *          own (within the pixel's level-of-detail depth window and up to its
 *          depth + eta), repeats each voxel's Alg. 1 decision and adds the vote
 *          with an atomic when the decision picks this pixel.  Pinhole maps only
 *          (TGV_ERR_UNSUPPORTED otherwise); the bounding box of a level's active
 *          bricks is indexed densely (at most 2^28 brick cells). */
enum { TGV_HIST_GATHER = 0, TGV_HIST_SCATTER = 1 };

typedef struct tgv_domain tgv_domain; /* opaque, library-owned */

/* Solver parameters (Eq. 2 with the primal-dual step sizes of Sec. 3.2).
 * Defaults (tgv_default_params): nbins 8 (Alg. 1), alpha1 1, alpha0 2, lambda 1,
 * tau = sigma = 0.2 (tau*sigma*24 < 1: ||K||^2 <= 24 for the forward/backward
 * difference operators), FP32 storage, clamp_u 1, endpoint centres, box_v 2,
 * paired iteration kernel, x_run 0 (automatic), gather-form histograms, default
 * wait budget, wait_test 0. */
typedef struct {
    int32_t nbins;       /* histogram bins, 2..16 */
    float alpha1;        /* weight of |grad u - v| */
    float alpha0;        /* weight of |E(v)| */
    float lambda;        /* weight of the histogram data term */
    float tau;           /* primal step */
    float sigma;         /* dual step */
    int32_t storage;     /* TGV_STORAGE_* */
    int32_t clamp_u;     /* 1: project u onto [-1, 1] after the prox */
    int32_t centres;     /* TGV_CENTRES_* */
    float box_v;         /* bound B_v on |v_a| used by the duality gap */
    int32_t iter_kernel; /* TGV_ITER_* form of the fused iteration kernel */
    int32_t x_run;       /* PAIRED form: work items per run, 0..64.  A CTA takes runs of
                          * consecutive items, so x-neighbouring bricks pass their face
                          * duals through shared memory; results do not depend on it.
                          * 0 = chosen from the item and SM counts, 1 = no runs. */
    int32_t hist_form;   /* TGV_HIST_* form of the histogram kernel */
    int64_t wait_cycles; /* budget of each bounded device-side wait of the PAIRED and PIPELINED
                          * iteration kernels (a CTA waiting for its bulk copies), in SM clock
                          * cycles; 0 = 2e9 (about one second).  A wait that runs out sets the
                          * domain's error flag: the next call that synchronises returns
                          * TGV_ERR_TIMEOUT and every later call TGV_ERR_STATE.  After giving up,
                          * a CTA still waits for its own copies in flight with the default budget,
                          * whatever this value, so none lands in released shared memory. */
    int32_t wait_test;   /* testing only, 0 in normal use.  1: the first wait of every CTA of the
                          * PAIRED kernel targets a barrier that no copy completes, so it runs out
                          * after wait_cycles (a way to exercise the timeout path without a fault) */
} tgv_params;

/* One level of a domain (all arrays host memory, copied at creation).
 *  origin, h: voxel grid of this level; radius: the voxel radius r of Alg. 1
 *  (r <= 0 selects h/2).  brick_coords: 3*nbricks int32 (x, y, z) of the
 *  active bricks, no duplicates.  frozen_coords: 3*nfrozen int32 of frozen
 *  bricks (disjoint from the active ones).  frozen_u: 512*nfrozen floats,
 *  frozen_v: 3*512*nfrozen floats laid out [brick][component][512]; either may
 *  be NULL (zeros, or filled later by tgv_prolong). */
typedef struct {
    double origin[3];
    double h;
    double radius;
    int64_t nbricks;
    const int32_t* brick_coords;
    int64_t nfrozen;
    const int32_t* frozen_coords;
    const float* frozen_u;
    const float* frozen_v;
} tgv_level_desc;

/* Depth-map camera (Sec. 3.1 depth maps, Sec. 3.4 LIDAR scans).  Frame
 * Xc = R (X - C), R row-major; pixel (i, j) covers [i, i+1) x [j, j+1).
 * NaN, inf and values <= 0 in a map mark pixels without a sample.
 *  TGV_PINHOLE: rows of R = right, down, forward; x = fx Xc/Zc + cx,
 *    y = fy Yc/Zc + cy (Zc > 0); maps hold the camera-frame z-depth of the
 *    observed point; a = depth - Zc; projected voxel diameter fx 2r / Zc.
 *  TGV_SPHERICAL (a LIDAR scan as a spherical depth map): rows of R = the
 *    scanner's x, y, z (z up); range rho = |Xc|, azimuth phi = atan2(Yc, Xc)
 *    in (-pi, pi], elevation theta = atan2(Zc, |(Xc, Yc)|) in [-pi/2, pi/2];
 *    x = fx phi + cx, y = cy - fy theta (fx, fy pixels per radian: a full
 *    scan of W x H has fx = W / (2 pi), cx = W / 2, fy = H / pi, cy = H / 2);
 *    maps hold the range of the observed point; a = depth - rho; projected
 *    voxel diameter fx 2r / rho.  The angles are evaluated in FP32 with one
 *    rounding per operation by the arctangent polynomial of Abramowitz &
 *    Stegun 4.4.49 (|error| <= 2e-8 rad on [0, 1]) after reducing the ratio
 *    min/max of the two arguments to [0, 1]; the exact step order is listed
 *    in tgv_hist.cu, so the pixel decision is reproducible bit for bit.
 * Votes: 1 per map, or 5 for noise-free LIDAR scans (Sec. 3.4). */
typedef struct {
    double fx, fy, cx, cy;
    double R[9];
    double C[3];
    int32_t width, height;
    int32_t model;
} tgv_camera;

/* Fills *out with the defaults listed at tgv_params. */
TGV_API tgv_status tgv_default_params(tgv_params* out);

/* Creates a domain of nlevels levels (level 0 coarsest).  Allocates all device
 * state on the current device; u, v, p, q and the histograms start at zero.
 * stream: a cudaStream_t (NULL = legacy default stream) used for every call.
 * Errors: INVALID_ARG (bad sizes, duplicate or overlapping bricks, nbins out of
 * range, unknown storage), OUT_OF_MEMORY, CUDA. */
TGV_API tgv_status tgv_create_domain(const tgv_level_desc* levels, int32_t nlevels, const tgv_params* prm,
                             void* stream, tgv_domain** out);

/* Frees all device state.  NULL is ignored. */
TGV_API void tgv_destroy_domain(tgv_domain* d);

/* Alg. 1 (Sec. 3.4) for one depth map: builds the map's mipmap pyramid on the
 * device (each coarser pixel = minimum of its valid children) and adds `vote`
 * (1, or 5 for noise-free LIDAR) to bin
 *   floor(((clamp(a/delta, -1, 1) + 1)/2) * nbins)   (clamped to nbins-1)
 * of every voxel whose centre projects to a valid pixel at its level of
 * detail and has a >= -eta (a = depth minus the voxel's z-depth, or range for
 * a spherical map), with delta = 6r, eta = 3 delta (Sec. 3.1).  The decision
 * is taken in FP32 with one rounding per operation.
 * depth_dev: device pointer, height rows of pitch_elems floats.
 * Errors: INVALID_ARG (level, camera, pitch < width, NULL), BUDGET (a voxel
 * count could pass 65535: counts are stored as 16-bit integers), CUDA. */
TGV_API tgv_status tgv_accumulate_depthmap(tgv_domain* d, int32_t level, const tgv_camera* cam,
                                   const float* depth_dev, int64_t pitch_elems, uint32_t vote);

/* Same as tgv_accumulate_depthmap for nmaps maps of one size in one pass:
 * map m starts at depth_dev + m * map_stride_elems; cams[m] and votes[m]
 * (votes may be NULL: all 1) are host arrays.  Results equal nmaps single
 * calls in any order (integer counts). */
TGV_API tgv_status tgv_accumulate_depthmaps(tgv_domain* d, int32_t level, const tgv_camera* cams, int32_t nmaps,
                                    const float* depth_dev, int64_t pitch_elems, int64_t map_stride_elems,
                                    const uint32_t* votes);

/* Runs `iterations` primal-dual iterations (Sec. 3.2; Chambolle-Pock order,
 * theta = 1) of Eq. 2 on one level:
 *   p <- proj_{|p|<=alpha1}(p + sigma (grad ubar - vbar))
 *   q <- proj_{|q|_F<=alpha0}(q + sigma E(vbar))
 *   u+ <- clamp(prox_{tau lambda hist}(u + tau div1 p)),  v+ <- v + tau (p + div2 q)
 *   ubar <- 2u+ - u,  vbar <- 2v+ - v
 * with forward differences for grad, backward differences for E (Eq. 3) and
 * their exact negative adjoints; frozen bricks stay fixed (Sec. 4.5).
 * energy_gap_out: NULL, or 4 doubles receiving (energy, dual value, gap,
 * certified) after the last iteration (see tgv_energy); a non-NULL pointer
 * synchronises the stream.  Errors: INVALID_ARG, STATE, CUDA. */
TGV_API tgv_status tgv_solve(tgv_domain* d, int32_t level, int32_t iterations, double* energy_gap_out);

/* Same as tgv_solve, run as a CUDA graph: the first call with a given
 * iteration count, starting ping-pong parity and work list launches its
 * kernels one by one and captures them into a graph; later matching calls
 * replay that graph with one launch.  Needs a non-NULL stream at creation
 * (UNSUPPORTED otherwise).  Graphs are freed with the domain. */
TGV_API tgv_status tgv_solve_graph(tgv_domain* d, int32_t level, int32_t iterations, double* energy_gap_out);

/* Persistent batched solve of independent chunks in one launch (Sec. 4.3: the treetop's
 * parts are solved independently; Sec. 4.5: each with its border cubes frozen).
 * Level `level` holds nchunks chunks: chunk c is the active bricks [first[c], first[c+1])
 * (host array of nchunks + 1 ascending brick indices; active bricks outside every chunk
 * keep their state); no face or edge link may join bricks of two chunks.  Chunk c runs
 * iterations[c] (host, >= 0) iterations of tgv_solve's scheme, and its result equals the
 * chunk solved alone by tgv_solve with the PAIRED kernel, bit for bit.
 * One persistent kernel: CTAs take tickets from a counter -- a ticket is a run of
 * run_length consecutive bricks of one chunk in one iteration, handed out iteration by
 * iteration -- and before a run wait (bounded by tgv_params.wait_cycles) at the chunk's
 * barrier until every run of the chunk's previous iteration has completed.  A CTA takes a
 * ticket only when its previous run is done, and a run waits only on smaller tickets, so
 * no wait depends on CTAs that are not running.  A wait that runs out makes the next
 * synchronising call return TGV_ERR_TIMEOUT.
 * run_length: 1..64 bricks, 0 = 16.  With a non-NULL stream the first call with a given
 * chunk table, iteration counts, run length and current ping-pong copy captures its
 * launches into a CUDA graph that later identical calls replay (up to 16 plans per level
 * are kept; they are freed with the domain).  Afterwards every chunk's ubar, vbar, p, q
 * are in the level's current copy.  Does not synchronise.
 * Errors: INVALID_ARG (ranges, a link between two chunks, a work list set), UNSUPPORTED
 * (levels of 2^31 bricks, a chunk with iterations x runs >= 2^31), OUT_OF_MEMORY, STATE,
 * CUDA. */
TGV_API tgv_status tgv_solve_chunks(tgv_domain* d, int32_t level, int32_t nchunks, const int64_t* first,
                                    const int32_t* iterations, int32_t run_length);

/* Restricts later iterations and energy evaluations of a level to the listed
 * active bricks (host or device int32 array of n distinct indices in [0,
 * nbricks)); bricks = NULL or n < 0 restores "every active brick".  Bricks
 * outside the list keep their state; none of them may be a face or edge
 * neighbour of a listed brick (the intended use: one level holding several
 * separated chunks, some of which are finished).  Errors: INVALID_ARG. */
TGV_API tgv_status tgv_set_work_list(tgv_domain* d, int32_t level, const int32_t* bricks, int64_t n);

/* Energy of Eq. 2 on the level (FP64 accumulation of FP32 per-voxel terms,
 * fixed-order deterministic reduction) and the value of the dual problem
 * with u in [-1, 1] and |v_a| <= box_v:
 *   out[0] = alpha1 sum|grad u - v| + alpha0 sum|E v|_F + lambda sum_x sum_b h_b|u - c_b|
 *   out[1] = <k0,(p,q)> - sum_x phi*_x(div1 p) - box_v |p + div2 q|_1
 *   out[2] = out[0] - out[1]  (>= 0 when out[3] = 1)
 *   out[3] = 1 if every |v_a| <= box_v, else 0
 * (k0 = the frozen-neighbour constants; phi*_x the conjugate of the clamped
 * data term.)  out: host, 4 doubles.  Synchronises the stream. */
TGV_API tgv_status tgv_energy(tgv_domain* d, int32_t level, double* out);

/* Copies a field of one level to `out` (host or device), voxel-major FP32,
 * count = number of active voxels * components of the field. */
TGV_API tgv_status tgv_extract_field(tgv_domain* d, int32_t level, int32_t field, float* out, int64_t count);

/* Overwrites a field of one level from `in` (host or device, same layout as
 * tgv_extract_field; values are rounded to the storage type). */
TGV_API tgv_status tgv_set_field(tgv_domain* d, int32_t level, int32_t field, const float* in, int64_t count);

/* Copies the histograms of one level to `out` (host or device):
 * uint32 [voxel][nbins], count = active voxels * nbins. */
TGV_API tgv_status tgv_extract_histograms(tgv_domain* d, int32_t level, uint32_t* out, int64_t count);

/* Overwrites the histograms of one level from `in` (host or device, same
 * layout).  Errors: BUDGET if a count exceeds 65535. */
TGV_API tgv_status tgv_set_histograms(tgv_domain* d, int32_t level, const uint32_t* in, int64_t count);

/* Zeroes u, ubar, v, vbar, p, q of a level (frozen bricks keep their values);
 * clear_hist != 0 also zeroes its histograms. */
TGV_API tgv_status tgv_reset(tgv_domain* d, int32_t level, int32_t clear_hist);

/* Coarse-to-fine start of level from_level+1 (Sec. 4.5): every active and
 * frozen voxel of the fine level takes u from its parent voxel on level
 * from_level and v halved (the index spacing halves); ubar = u, vbar = v,
 * p = q = 0.  Requires equal origins and h_fine = h_coarse / 2.  Fine voxels
 * without an active parent get u = v = 0.  Errors: INVALID_ARG. */
TGV_API tgv_status tgv_prolong(tgv_domain* d, int32_t from_level);

/* Waits for all work queued on the domain's stream. */
TGV_API tgv_status tgv_synchronize(tgv_domain* d);

/* Device bytes held by the domain (state, tables, scratch). */
TGV_API int64_t tgv_domain_bytes(const tgv_domain* d);

/* Number of active voxels of a level (0 for a bad level). */
TGV_API int64_t tgv_level_voxels(const tgv_domain* d, int32_t level);

/* Number of kernels this library launched on the domain so far. */
TGV_API int64_t tgv_launch_count(const tgv_domain* d);

/* Marching cubes (Sec. 4.6): the zero level set of level `level`'s u as a
 * welded triangle mesh, kept in library-owned device memory until the next
 * extraction or tgv_destroy_domain; writes its vertex and triangle counts.
 *  Cells: cubes of 8 voxel centres, one per voxel g of an active brick (its
 *  lower corner), extracted when all 8 corners exist (active or frozen bricks).
 *  Corner inside when u < 0.  Vertices: the zero crossing on each edge with
 *  ends of different sides, t = u_p / (u_p - u_q), world coordinates
 *  origin + (idx + 0.5 (+ t along the edge)) h, FP32 with one rounding per
 *  operation.  Per cell, each face joins the crossing where its boundary
 *  (counter-clockwise seen from outside the cell) enters the inside region to
 *  the next one where it leaves; with four crossings, the face sum
 *  ((u_a + u_b) + (u_c + u_d)) of its corners in cell order picks the next
 *  (>= 0) or the previous (< 0) exit, so both cells of a face agree.  The joins
 *  form loops, counter-clockwise seen from u >= 0 (triangle normals point to
 *  u >= 0), each triangulated by the minimum-area dynamic programme (FP32, ties
 *  to the smallest split) without chords along a cell face; a loop with no such
 *  triangulation is fanned around its centroid (one extra vertex per cell).
 *  The mesh of a closed zero set inside the domain is closed and consistently
 *  oriented.
 *  Vertex order: increasing id (4 slot + axis for a crossing on the edge from
 *  voxel slot along axis, 4 slot + 3 for a cell's centroid; slot = brick * 512
 *  + local, frozen brick f at brick index nbricks + f); triangles in cell order.
 * Errors: INVALID_ARG, UNSUPPORTED (more than 2^31 vertices or 2^32 ids),
 * OUT_OF_MEMORY, CUDA.  Synchronises the stream. */
TGV_API tgv_status tgv_extract_mesh(tgv_domain* d, int32_t level, int64_t* nverts, int64_t* ntris);

/* Copies the last extracted mesh: verts = 3 * nverts floats (x, y, z),
 * tris = 3 * ntris int32 vertex indices (host or device pointers).  The counts
 * must equal those tgv_extract_mesh returned (INVALID_ARG otherwise; STATE if
 * there is no mesh).  Synchronises the stream. */
TGV_API tgv_status tgv_copy_mesh(tgv_domain* d, float* verts, int64_t nverts, int32_t* tris, int64_t ntris);

/* ---------------------------------------------------------------------------
 * Joint solve of all levels of a domain on their composite grid (Sec. 3.3: in
 * a 2:1-balanced octree a cube has up to four neighbours over a face; Eq. 2-3,
 * Sec. 3.2), instead of one level after another with frozen shells.
 * Leaves: voxels of level l in an active brick whose 8 children are not in an
 * active brick of level l+1 (levels nested 2:1, as tgv_octree_build makes
 * them).  Every difference is a unit index step, as on a single level; for
 * leaf x and axis a the +a neighbours are the same-level leaf x + e_a, else
 * the coarser leaf containing that position, else the 4 children of the
 * refined voxel there on the face next to x, else none (likewise -a):
 *   (G_a u)(x) = mean(u over +a neighbours) - u(x),
 *   (B_a w)(x) = w(x) - mean(w over -a neighbours)   (0 without neighbours),
 *   E(v)_ab = (B_a v_b + B_b v_a) / 2, div1 = -sum_a G_a^T,
 *   (div2 q)_b = -sum_a B_a^T q_ab (exact negative adjoints);
 * the Chambolle-Pock iteration of tgv_solve with the domain's parameters, each
 * leaf using the histogram of its own level; outer boundaries Neumann (frozen
 * bricks are not used).  State in FP32 whatever the domain's storage; u and
 * ubar start from the levels' u, v, vbar, p, q from 0.  Leaf order: level by
 * level, brick order, local voxel index.
 * ------------------------------------------------------------------------- */
typedef struct tgv_composite tgv_composite; /* opaque, library-owned */

/* Builds the composite of every level of d (host lists + device state; the
 * histograms must be accumulated).  Keeps a reference to d (destroy the
 * composite first).  Errors: INVALID_ARG (levels not 2:1 nested), STATE,
 * OUT_OF_MEMORY, UNSUPPORTED (2^31 leaves), CUDA.  Synchronises. */
TGV_API tgv_status tgv_composite_create(tgv_domain* d, tgv_composite** out);
/* `iterations` joint iterations (two kernels each) on d's stream. */
TGV_API tgv_status tgv_composite_solve(tgv_composite* c, int32_t iterations);
TGV_API int64_t tgv_composite_leaves(const tgv_composite* c);
/* Leaves of one level (-1 for a bad level). */
TGV_API int64_t tgv_composite_level_leaves(const tgv_composite* c, int32_t level);
/* Copies u of every leaf (count = leaves, host or device).  Synchronises. */
TGV_API tgv_status tgv_composite_extract(tgv_composite* c, float* u_out, int64_t count);
/* Writes each leaf's u into its level's u (refined voxels keep theirs), so
 * tgv_extract_field / tgv_extract_mesh see the joint result.  Synchronises. */
TGV_API tgv_status tgv_composite_scatter(tgv_composite* c);
TGV_API int64_t tgv_composite_launch_count(const tgv_composite* c);

/* Treetop of the composite grid (Sec. 4.3): the leaves are the octree's leaf
 * cubes; in Z-order (Morton order of their lower corners) the leaves under any
 * octree node are consecutive, and the treetop is the smallest rooted subtree
 * whose leaf nodes each hold fewer than max_cubes leaf cubes.  The root is the
 * cube [0, 2^root_bits)^3 in voxel units of the finest level (for levels from
 * tgv_octree_build: root_bits = dmax + 3, and node depths are octree depths);
 * a node of depth k is an aligned cube of 2^(root_bits - k) finest voxels per
 * axis, with code = the top 3k bits of its cubes' Morton codes.  Nodes holding
 * no leaf are not parts.  A part is a leaf node of the treetop: the leaves
 * under it form the range [first, last] of the Z-ordered leaves (the paper's
 * two indices per treetop leaf, the unit of independent work).  Writes the
 * number of parts; parts come in Z-order.
 * Errors: INVALID_ARG (root_bits outside 1..21, max_cubes < 2, a leaf with a
 * negative coordinate or outside the root cube), UNSUPPORTED (3 root_bits +
 * ceil(log2 leaves) > 64), OUT_OF_MEMORY, STATE, CUDA.  Synchronises. */
TGV_API tgv_status tgv_composite_treetop(tgv_composite* c, int32_t root_bits, int64_t max_cubes, int64_t* nparts);
/* Copies the last treetop: per part its depth, code, first and last Z-index
 * (host arrays of nparts entries, each nullable), and per leaf (composite
 * order) its part index (leaves int32, host or device, nullable).  STATE
 * without a treetop.  Synchronises. */
TGV_API tgv_status tgv_composite_treetop_parts(tgv_composite* c, int32_t* depth, uint64_t* code, int64_t* first,
                                               int64_t* last, int32_t* leaf_part);
TGV_API void tgv_composite_destroy(tgv_composite* c);

/* ---------------------------------------------------------------------------
 * Brick domains from depth maps (Sec. 3.3 Eq. 4, Sec. 4.1-4.2; in memory, one
 * GPU).  Every valid pixel is a sample: a pinhole map's z-depth, or a
 * spherical map's range along the pixel's direction (azimuth phi =
 * (i + 0.5 - cx) / fx, elevation theta = (cy - (j + 0.5)) / fy; direction
 * (cos theta cos phi, cos theta sin phi, sin theta) in the scanner's axes, with
 * sin and cos evaluated in FP32 by the library's own reduction by pi/2 and
 * Taylor polynomials, |error| < 1.2e-7), unprojected to X; radius r = half the
 * mean distance to the points of its valid 4-neighbours (left, right, up, down;
 * a scan's azimuth seam is not crossed).  Eq. 4 puts it in the cube of
 * depth d with 0.75 r <= r_root 2^-d < 1.5 r (r_root = root_edge / 2): the
 * smallest d in [depth_min, depth_max] with r_root 2^-d < 1.5 r (depth_max if
 * none), cube q = floor(((X - root_min) / root_edge) 2^d), samples outside the
 * root dropped; all in FP32 with one rounding per operation (order in
 * tgv_octree.cu).  Level l = d - depth_min: voxel edge root_edge / 2^d, origin
 * root_min; active bricks = the occupied cubes' q >> 3, dilated `band` times
 * by their 26 neighbours; then, finest first, level l-1 gains the parents
 * (b >> 1) of level l's bricks dilated once (2:1 balance: each finer level is
 * wrapped by a shell of the next coarser level); frozen bricks of level l > 0
 * = the non-active 26-neighbours of its active bricks.  Neighbours stay inside
 * the root.  Bricks are listed in Morton (Z-curve) order.  The levels feed
 * tgv_create_domain for a coarse-to-fine solve (frozen values by tgv_prolong).
 * ------------------------------------------------------------------------- */
typedef struct {
    double root_min[3];
    double root_edge;   /* root cube [root_min, root_min + root_edge)^3 */
    int32_t depth_min;  /* >= 3 (one brick = 8 cubes per axis) */
    int32_t depth_max;  /* depth_min..21 */
    int32_t band;       /* dilation rings of the occupied bricks, 0..8 */
} tgv_octree_cfg;

typedef struct tgv_octree tgv_octree; /* opaque, library-owned (host memory) */

/* Builds the levels from nmaps maps of one size, pinhole or spherical (map m at
 * depth_dev + m * map_stride_elems, rows of pitch_elems floats, device memory;
 * cams on the host) on `stream`.  Errors: INVALID_ARG (also an unknown camera
 * model), OUT_OF_MEMORY, BUDGET (the device hash set could not hold the
 * bricks), CUDA.  Synchronises the stream. */
TGV_API tgv_status tgv_octree_build(const tgv_octree_cfg* cfg, const tgv_camera* cams, int32_t nmaps,
                                    const float* depth_dev, int64_t pitch_elems, int64_t map_stride_elems,
                                    void* stream, tgv_octree** out);
TGV_API int32_t tgv_octree_levels(const tgv_octree* o);
/* Number of samples that fell inside the root. */
TGV_API int64_t tgv_octree_samples(const tgv_octree* o);
/* Counts, origin (3 doubles) and voxel edge of a level (any output may be NULL). */
TGV_API tgv_status tgv_octree_level(const tgv_octree* o, int32_t level, int64_t* nactive, int64_t* nfrozen,
                                    double* origin, double* h);
/* Copies a level's brick coordinates (3 int32 per brick) into host arrays sized
 * from tgv_octree_level. */
TGV_API tgv_status tgv_octree_bricks(const tgv_octree* o, int32_t level, int32_t* active, int32_t* frozen);
TGV_API void tgv_octree_destroy(tgv_octree* o);

/* Run length the paired iteration kernel chooses when tgv_params.x_run is 0
 * (host only; no device work).  The iteration is Eq. 2-3 whatever the choice;
 * it only sets how many consecutive work items a CTA takes in a row, trading
 * x-face halo work saved by hand-overs against load balance and the L2 reuse
 * of neighbours' face layers (a cost model over the level's links).
 *  nbr:   host, nbricks x 12 neighbour rows in the library's layout (faces +x,
 *         -x, +y, -y, +z, -z, then the six mixed-sign edges; -1 none, >= nbricks
 *         frozen), as built for the level;
 *  work:  host list of nwork distinct active bricks, or NULL for all bricks in order;
 *  slots: resident CTAs of the kernel (CTAs per SM x SMs), > 0;
 *  storage: TGV_STORAGE_*.
 * Writes 1..16 to *run_length.  TGV_ERR_INVALID_ARG on bad sizes or a work
 * list entry that is out of range or repeated. */
TGV_API tgv_status tgv_pair_run_length(const int32_t* nbr, int64_t nbricks, const int32_t* work, int64_t nwork,
                                       int64_t slots, int32_t storage, int32_t* run_length);

/* ---------------------------------------------------------------------------
 * Energy / gap without any allocation.
 *
 * The paper has no counterpart to this call; it exists for callers that may
 * not allocate device memory: a serving process that reserved all of its HBM
 * up front for admitted requests, or a host framework whose own memory pool
 * owns the device (a stray cudaMalloc there can fail for lack of unreserved
 * memory, and cudaMalloc/cudaFree may synchronise the device and stall the
 * other streams).  Such a caller keeps a level's state in buffers it owns,
 * laid out as described by tgv_state_view, and gets the same four numbers as
 * tgv_energy.
 *
 * The reduction scratch is a fixed array inside this library (on every GPU
 * that loads the library, held until the process exits), so the call
 * allocates nothing and frees nothing.  It holds one set of partial sums per
 * CTA of the energy kernel (sixteen CTAs per SM), so any number of active bricks
 * fits.  Consequences:
 *  - every call on a device uses the same scratch: calls whose device work
 *    overlaps (different streams, or other host threads) race and may return
 *    wrong numbers; serialise them (one stream, or wait for the previous
 *    call);
 *  - the first call on a device looks up the scratch array's device address
 *    (once per device, with that device current); make that first call before
 *    any stream capture begins;
 *  - that address belongs to the device's context of the time: after a
 *    cudaDeviceReset (or anything else that destroys the device's primary
 *    context) in the same process it is stale, so do not call this entry point
 *    on a device reset since its first call.
 * `stream`: the cudaStream_t to run on (NULL = legacy default stream); the
 * call waits for its own work.  `out`: 4 doubles, host or device memory,
 * receiving the same values as tgv_energy.  Errors: INVALID_ARG (null
 * pointers, bad parameters), BUDGET (a device with more than 256 SMs), CUDA.
 * ------------------------------------------------------------------------- */

/* One level's state in device memory owned by the caller (the library's
 * layout: brick-major, 512 voxels per brick, local index i + 8j + 64k;
 * active bricks first, then frozen ones). */
typedef struct {
    int64_t nbricks;        /* active bricks (nb) */
    int64_t nall;           /* active + frozen bricks */
    const float* u;         /* [nall][512] */
    const void* v;          /* [nall][3][512], storage type of the params */
    const void* p;          /* [nb][3][512] */
    const void* q;          /* [nb][6][512]: xx, yy, zz, xy, xz, yz */
    const uint32_t* hist;   /* [nb][(nbins+1)/2][512]: bin 2k in the low 16 bits, 2k+1 in the high */
    const int32_t* nbr;     /* [nb][12] neighbour brick per slot, offsets (+x), (-x), (+y), (-y), (+z), (-z),
                               (-x,+y), (-x,+z), (+x,-y), (-y,+z), (+x,-z), (+y,-z); -1 = none,
                               >= nbricks = frozen (only the six faces are read here) */
} tgv_state_view;

TGV_API tgv_status tgv_energy_noalloc(const tgv_state_view* s, const tgv_params* prm, void* stream, double* out);

/* ---------------------------------------------------------------------------
 * Serving: chunk-solve requests with continuous batching.
 *
 * A request is one independent part of a domain (Sec. 4.3 treetop leaves:
 * the parts are solved independently, their border cubes frozen, Sec. 4.5):
 * a set of active bricks, its frozen shell and its histograms.  A server
 * keeps every admitted request's state resident in one device arena whose
 * capacity is fixed at creation (the HBM budget), and advances all running
 * requests together: each fused iteration launch covers the work list of
 * every running request, so requests that arrive while others are running
 * join the next launch, and finished ones leave it.  A request's result is
 * the same as solving it alone (no link ever leaves a request).
 * All requests of a server share nbins and the other parameters.
 * ------------------------------------------------------------------------- */
typedef struct tgv_server tgv_server;

typedef struct {
    int64_t capacity_bricks;  /* active bricks the arena holds */
    int64_t capacity_frozen;  /* frozen bricks the arena holds */
    int64_t staging_bytes;    /* pinned host staging for inputs (<= 0: 256 MiB) */
} tgv_server_cfg;

/* Creates a server and allocates its arena on the current device.  stream:
 * a non-NULL cudaStream_t for all of its work.  Errors: INVALID_ARG,
 * OUT_OF_MEMORY, CUDA. */
TGV_API tgv_status tgv_server_create(const tgv_server_cfg* cfg, const tgv_params* prm, void* stream,
                                     tgv_server** out);

/* Admits a request: chunk = its active bricks and frozen shell (frozen_u /
 * frozen_v as in tgv_level_desc; origin, h, radius unused), hist = uint32
 * [voxel][nbins] counts (host or device; device memory must stay valid until
 * the server's stream reaches this call; counts above 65535 are not
 * allowed), `iterations` primal-dual iterations from u = v = p = q = 0.
 * Returns a ticket.  Errors: BUDGET (not enough free arena space right now:
 * retry after extracting finished requests), INVALID_ARG (a request larger
 * than the whole arena, bad bricks), CUDA. */
TGV_API tgv_status tgv_server_submit(tgv_server* s, const tgv_level_desc* chunk, const uint32_t* hist,
                                     int32_t iterations, uint64_t* ticket);

/* Queues up to max_iterations fused iterations over every running request,
 * stopping early at the first iteration after which some request has run
 * its count; *finished (nullable) receives how many requests finished.  Does
 * not wait for the device. */
TGV_API tgv_status tgv_server_step(tgv_server* s, int32_t max_iterations, int32_t* finished);

/* *done = 1 once the request's iterations have all been queued. */
TGV_API tgv_status tgv_server_poll(tgv_server* s, uint64_t ticket, int32_t* done);

/* Copies a finished request's u (voxel order of its chunk, count = its
 * active voxels) to u_out (host or device), waiting only for that request's
 * work, and releases its arena space and ticket. */
TGV_API tgv_status tgv_server_extract(tgv_server* s, uint64_t ticket, float* u_out, int64_t count);

/* Free active-brick capacity, running requests, voxel-updates queued so far. */
TGV_API int64_t tgv_server_free_bricks(const tgv_server* s);
TGV_API int64_t tgv_server_running(const tgv_server* s);
TGV_API int64_t tgv_server_voxel_updates(const tgv_server* s);

/* Message of the last failure on the server. */
TGV_API const char* tgv_server_last_error(const tgv_server* s);

/* Waits for all queued work of the server. */
TGV_API tgv_status tgv_server_synchronize(tgv_server* s);

TGV_API void tgv_server_destroy(tgv_server* s);

TGV_API const char* tgv_status_string(tgv_status s);
TGV_API const char* tgv_last_error(const tgv_domain* d);

#ifdef __cplusplus
}
#endif

#endif /* TGV_H_ */
