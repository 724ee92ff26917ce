/*
 * FP64 CPU oracle for the histogram + TGV primal-dual path of
 * "Out-of-Core Surface Reconstruction via Global TGV Minimization" (arXiv 2107.14790).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline / reference legs may load this library.  The product path (the
 * CUDA library in paper_2107_14790_b300/) never calls it, and this file shares
 * no code, header, table or helper with that library.
 *
 * Plain, slow, obviously correct loops.  Each function names the passage it
 * follows.  Where the paper is silent, the reading taken is stated inline.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fopenmp -shared -fPIC
 *   -ffp-contract=off is required: the histogram decision (Alg. 1) is taken in
 *   FP32 with one rounding per listed operation, exactly like the kernel.
 *
 * Parity status: every function here is pinned by a test in tests/test_oracle_*.py
 * (closed forms, invariants, brute force); none is "parity unpinned".  The
 * converged field is pinned only against the sphere's geometry.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_BRICK 8
#define ORC_BVOX 512

/* ======================================================================== */
/* Depth pyramid (Sec. 3.4: depth maps get mipmap pyramids; Alg. 1 projects  */
/* into the pyramid level matching the voxel's projected size).              */
/* Reading: level l+1 has ceil(W_l/2) x ceil(H_l/2) pixels; each pixel is    */
/* the minimum of its existing, valid children; invalid if none is valid.    */
/* Levels run up to Lmax = floor(log2(max(W, H))).  Invalid = NaN, inf, <=0. */
/* ======================================================================== */
int orc_pyramid_nlevels(int W, int H)
{
    int m = W > H ? W : H;
    int L = 0;
    while ((1 << (L + 1)) <= m) L++;
    return L + 1;
}

/* dims[2*l], dims[2*l+1] = width, height of level l; offs[l] = element offset. */
int64_t orc_pyramid_layout(int W, int H, int32_t* dims, int64_t* offs)
{
    int n = orc_pyramid_nlevels(W, H);
    int64_t off = 0;
    int w = W, h = H;
    for (int l = 0; l < n; ++l) {
        dims[2 * l] = w;
        dims[2 * l + 1] = h;
        offs[l] = off;
        off += (int64_t)w * h;
        w = (w + 1) / 2;
        h = (h + 1) / 2;
    }
    return off;
}

static int orc_valid_depth(float d) { return isfinite(d) && d > 0.0f; }

void orc_build_pyramid(const float* depth, int W, int H, int64_t pitch, float* pyr)
{
    int32_t dims[64];
    int64_t offs[32];
    int n = orc_pyramid_nlevels(W, H);
    orc_pyramid_layout(W, H, dims, offs);
    for (int j = 0; j < H; ++j)
        for (int i = 0; i < W; ++i) {
            float d = depth[(int64_t)j * pitch + i];
            pyr[(int64_t)j * W + i] = orc_valid_depth(d) ? d : NAN;
        }
    for (int l = 1; l < n; ++l) {
        int wp = dims[2 * (l - 1)], hp = dims[2 * (l - 1) + 1];
        int w = dims[2 * l], h = dims[2 * l + 1];
        const float* src = pyr + offs[l - 1];
        float* dst = pyr + offs[l];
        for (int j = 0; j < h; ++j)
            for (int i = 0; i < w; ++i) {
                float best = NAN;
                for (int dj = 0; dj < 2; ++dj)
                    for (int di = 0; di < 2; ++di) {
                        int ci = 2 * i + di, cj = 2 * j + dj;
                        if (ci >= wp || cj >= hp) continue;
                        float c = src[(int64_t)cj * wp + ci];
                        if (isnan(c)) continue;
                        if (isnan(best) || c < best) best = c;
                    }
                dst[(int64_t)j * w + i] = best;
            }
    }
}

/* ======================================================================== */
/* Algorithm 1 (add_to_voxel_histograms), one voxel and one depth map.       */
/*                                                                          */
/* The decision is taken in FP32, one rounding per operation, in this order  */
/* (the kernel takes the same decision in the same precision):               */
/*   X   = o + ((float)idx + 0.5) * h            per axis                     */
/*   d   = X - C;  Xc = (R0 d0 + R1 d1) + R2 d2  (rows of R), likewise Yc, Zc */
/*   in front of the camera iff Zc > 0                                        */
/*   x   = (fx*Xc)/Zc + cx,  y = (fy*Yc)/Zc + cy                              */
/*   fp  = (fx*(2r))/Zc    projected voxel diameter in level-0 pixels         */
/*   LOD = largest l in [0, Lmax] with 2^l <= max(1, fp)   (exact compares)   */
/*   pixel at LOD: (floor(x/2^l), floor(y/2^l)), must lie inside the level    */
/*   depth = pyramid[l][pixel]; invalid -> no vote                            */
/*   a = depth - Zc  (Alg. 1: depth minus distance; distance = z-depth)       */
/*   delta = 6 r, eta = 3 delta (Sec. 3.1);  a < -eta -> no vote              */
/*   a' = max(-1, min(1, a/delta));  bin = floor(((a'+1)/2) * n)              */
/*   bin = min(bin, n-1)   (reading: Alg. 1 gives bin = n at a' = +1)         */
/* Camera parameters arrive as FP64 and are rounded once to FP32.            */
/* Returns 1 and sets *bin when the map votes for the voxel, else 0.         */
/*                                                                          */
/* Spherical maps (LIDAR scans, Sec. 3.4), reading: the frame rows are the   */
/* scanner's x, y, z; the map stores the range of the observed point, and    */
/* the "distance" of Alg. 1 is the voxel centre's range rho = |Xc|:          */
/*   s2 = Xc*Xc + Yc*Yc;  rho = sqrt(s2 + Zc*Zc)  (requires rho > 0)         */
/*   azimuth phi = atan2(Yc, Xc), elevation theta = atan2(Zc, sqrt(s2))      */
/*   x = fx*phi + cx,  y = cy - fy*theta,  fp = (fx*(2r))/rho,  a = depth-rho */
/* with atan2 taken in FP32 by the arctangent polynomial of Abramowitz and   */
/* Stegun 4.4.49 (orc_atan2_as below), so both sides decide identically.     */
/* ======================================================================== */
typedef struct {
    float fx, fy, cx, cy, R[9], C[3];
    int W, H;
    int spherical;
} orc_cam32;

/* cam: 17 doubles (fx, fy, cx, cy, R row-major, C, model: 0 pinhole, 1 spherical) */
static orc_cam32 orc_cam_from_f64(const double* cam, int W, int H)
{
    orc_cam32 c;
    c.fx = (float)cam[0];
    c.fy = (float)cam[1];
    c.cx = (float)cam[2];
    c.cy = (float)cam[3];
    for (int k = 0; k < 9; ++k) c.R[k] = (float)cam[4 + k];
    for (int k = 0; k < 3; ++k) c.C[k] = (float)cam[13 + k];
    c.W = W;
    c.H = H;
    c.spherical = cam[16] == 1.0;
    return c;
}

/* atan2(y, x) in FP32 (every operation rounded to float, no contraction):
 * t = min(|x|,|y|) / max(|x|,|y|) in [0, 1]; arctan t by A&S 4.4.49,
 *   arctan t ~ t (1 + a2 t^2 + a4 t^4 + ... + a16 t^16),  |error| <= 2e-8,
 * the bracket evaluated by Horner in s = t^2 from a16 down to the constant 1;
 * then the octant: |y| > |x| -> pi/2 - r; x < 0 -> pi - r; y < 0 -> -r.
 * atan2(0, 0) = 0. */
float orc_atan2_as(float y, float x)
{
    static const float a[8] = {-0.3333314528f, 0.1999355085f, -0.1420889944f, 0.1065626393f,
                               -0.0752896400f, 0.0429096138f, -0.0161657367f, 0.0028662257f};
    float ax = fabsf(x), ay = fabsf(y);
    float big = ax > ay ? ax : ay, small = ax > ay ? ay : ax;
    if (big == 0.0f) return 0.0f;
    float t = small / big;
    float s = t * t;
    float p = a[7];
    for (int k = 6; k >= 0; --k) p = p * s + a[k];
    p = p * s + 1.0f;
    float r = t * p;
    if (ay > ax) r = 1.5707963267948966f - r;
    if (x < 0.0f) r = 3.14159265358979323846f - r;
    if (y < 0.0f) r = -r;
    return r;
}

static int orc_vote_f32(const orc_cam32* cam, const float* pyr, int nlev, const int32_t* dims,
                        const int64_t* offs, const float o[3], float h, float r, const int64_t idx[3],
                        int nbins, int* bin_out)
{
    float X[3], d[3];
    for (int a = 0; a < 3; ++a) {
        float t = (float)idx[a] + 0.5f;
        float m = t * h;
        X[a] = o[a] + m;
        d[a] = X[a] - cam->C[a];
    }
    const float* R = cam->R;
    float xc = R[0] * d[0] + R[1] * d[1];
    xc = xc + R[2] * d[2];
    float yc = R[3] * d[0] + R[4] * d[1];
    yc = yc + R[5] * d[2];
    float zc = R[6] * d[0] + R[7] * d[1];
    zc = zc + R[8] * d[2];
    float diam = r * 2.0f;
    float px, py, fp, dist;
    if (!cam->spherical) {
        if (!(zc > 0.0f)) return 0;
        px = (cam->fx * xc) / zc + cam->cx;
        py = (cam->fy * yc) / zc + cam->cy;
        fp = (cam->fx * diam) / zc;
        dist = zc;
    } else {
        float s2 = xc * xc + yc * yc;
        float rho = sqrtf(s2 + zc * zc);
        if (!(rho > 0.0f)) return 0;
        float phi = orc_atan2_as(yc, xc);
        float theta = orc_atan2_as(zc, sqrtf(s2));
        px = cam->fx * phi + cam->cx;
        py = cam->cy - cam->fy * theta;
        fp = (cam->fx * diam) / rho;
        dist = rho;
    }
    int L = 0;
    float p2 = 2.0f;
    while (L + 1 < nlev && p2 <= fp) {
        L++;
        p2 = p2 * 2.0f;
    }
    float scale = ldexpf(1.0f, -L);
    float xl = px * scale, yl = py * scale;
    int wl = dims[2 * L], hl = dims[2 * L + 1];
    if (!(xl >= 0.0f && xl < (float)wl)) return 0;
    if (!(yl >= 0.0f && yl < (float)hl)) return 0;
    int i = (int)floorf(xl), j = (int)floorf(yl);
    float depth = pyr[offs[L] + (int64_t)j * wl + i];
    if (isnan(depth)) return 0;
    float a = depth - dist;
    float delta = 6.0f * r;
    float eta = 3.0f * delta;
    if (a < -eta) return 0;
    float ac = a / delta;
    if (ac > 1.0f) ac = 1.0f;
    if (ac < -1.0f) ac = -1.0f;
    float t1 = ac + 1.0f;
    float t2 = t1 / 2.0f;
    float t3 = t2 * (float)nbins;
    int bin = (int)floorf(t3);
    if (bin > nbins - 1) bin = nbins - 1;
    *bin_out = bin;
    return 1;
}

/* Same decision in FP64 throughout (diagnostic: counts votes whose bin or
 * acceptance differs from the FP32 decision). */
static int orc_vote_f64(const double* cam, int L32, const float* pyr, const int32_t* dims,
                        const int64_t* offs, const double o[3], double h, double r, const int64_t idx[3],
                        int nbins, int* bin_out)
{
    double d[3];
    for (int a = 0; a < 3; ++a) d[a] = o[a] + ((double)idx[a] + 0.5) * h - cam[13 + a];
    const double* R = cam + 4;
    double xc = R[0] * d[0] + R[1] * d[1] + R[2] * d[2];
    double yc = R[3] * d[0] + R[4] * d[1] + R[5] * d[2];
    double zc = R[6] * d[0] + R[7] * d[1] + R[8] * d[2];
    double px, py, dist;
    if (cam[16] != 1.0) {
        if (!(zc > 0.0)) return 0;
        px = cam[0] * xc / zc + cam[2];
        py = cam[1] * yc / zc + cam[3];
        dist = zc;
    } else {
        dist = sqrt(xc * xc + yc * yc + zc * zc);
        if (!(dist > 0.0)) return 0;
        px = cam[0] * atan2(yc, xc) + cam[2];
        py = cam[3] - cam[1] * atan2(zc, sqrt(xc * xc + yc * yc));
    }
    int L = L32; /* use the FP32 LOD so the diagnostic isolates binning */
    double xl = ldexp(px, -L), yl = ldexp(py, -L);
    int wl = dims[2 * L], hl = dims[2 * L + 1];
    if (!(xl >= 0.0 && xl < wl && yl >= 0.0 && yl < hl)) return 0;
    int i = (int)floor(xl), j = (int)floor(yl);
    float depth = pyr[offs[L] + (int64_t)j * wl + i];
    if (isnan(depth)) return 0;
    double a = (double)depth - dist;
    double delta = 6.0 * r, eta = 3.0 * delta;
    if (a < -eta) return 0;
    double ac = fmax(-1.0, fmin(1.0, a / delta));
    int bin = (int)floor((ac + 1.0) / 2.0 * nbins);
    if (bin > nbins - 1) bin = nbins - 1;
    *bin_out = bin;
    return 1;
}

/* LOD the FP32 decision picks (for the FP64 diagnostic). */
static int orc_lod_f32(const orc_cam32* cam, int nlev, const float o[3], float h, float r, const int64_t idx[3])
{
    float d[3];
    for (int a = 0; a < 3; ++a) {
        float t = (float)idx[a] + 0.5f;
        float m = t * h;
        d[a] = (o[a] + m) - cam->C[a];
    }
    float zc = cam->R[6] * d[0] + cam->R[7] * d[1];
    zc = zc + cam->R[8] * d[2];
    float dist = zc;
    if (cam->spherical) {
        float xc = cam->R[0] * d[0] + cam->R[1] * d[1];
        xc = xc + cam->R[2] * d[2];
        float yc = cam->R[3] * d[0] + cam->R[4] * d[1];
        yc = yc + cam->R[5] * d[2];
        dist = sqrtf((xc * xc + yc * yc) + zc * zc);
    }
    float fp = (cam->fx * (r * 2.0f)) / dist;
    int L = 0;
    float p2 = 2.0f;
    while (L + 1 < nlev && p2 <= fp) {
        L++;
        p2 = p2 * 2.0f;
    }
    return L;
}

/*
 * Gather form of Alg. 1 over every voxel of a brick level for one depth map.
 *   bricks[3*b+a]: brick coordinates; voxel (i,j,k) of brick b has global index
 *   8*brick + (i,j,k) and flat id b*512 + i + 8 j + 64 k.
 *   hist: uint32 [nvox][nbins], incremented by `vote` in place.
 *   cam: 17 doubles (fx, fy, cx, cy, R row-major, C, model 0 pinhole / 1 spherical).
 *   r: voxel radius (Sec. 3.3, Eq. 5; reading: r = h/2 on a dense level).
 * Returns the number of votes cast; *ndiff64 (nullable) receives the number of
 * voxels where the FP64 decision differs from the FP32 one.
 */
int64_t orc_accumulate(int64_t nbricks, const int32_t* bricks, const double* origin, double h, double r,
                       const double* cam, int W, int H, const float* pyr, int nbins, uint32_t vote,
                       uint32_t* hist, int64_t* ndiff64)
{
    orc_cam32 c32 = orc_cam_from_f64(cam, W, H);
    int32_t dims[64];
    int64_t offs[32];
    int nlev = orc_pyramid_nlevels(W, H);
    orc_pyramid_layout(W, H, dims, offs);
    float o32[3] = {(float)origin[0], (float)origin[1], (float)origin[2]};
    float h32 = (float)h, r32 = (float)r;
    int64_t votes = 0, diffs = 0;
    for (int64_t b = 0; b < nbricks; ++b)
        for (int v = 0; v < ORC_BVOX; ++v) {
            int64_t idx[3] = {(int64_t)ORC_BRICK * bricks[3 * b + 0] + (v & 7),
                              (int64_t)ORC_BRICK * bricks[3 * b + 1] + ((v >> 3) & 7),
                              (int64_t)ORC_BRICK * bricks[3 * b + 2] + (v >> 6)};
            int bin = -1;
            int ok = orc_vote_f32(&c32, pyr, nlev, dims, offs, o32, h32, r32, idx, nbins, &bin);
            if (ok) {
                hist[(b * ORC_BVOX + v) * nbins + bin] += vote;
                votes++;
            }
            if (ndiff64) {
                int bin64 = -1, ok64 = 0;
                double zc_test;
                {
                    double d[3];
                    for (int a = 0; a < 3; ++a) d[a] = origin[a] + ((double)idx[a] + 0.5) * h - cam[13 + a];
                    zc_test = cam[10] * d[0] + cam[11] * d[1] + cam[12] * d[2];
                }
                if (zc_test > 0.0 || cam[16] == 1.0) {
                    int L = orc_lod_f32(&c32, nlev, o32, h32, r32, idx);
                    ok64 = orc_vote_f64(cam, L, pyr, dims, offs, origin, h, r, idx, nbins, &bin64);
                }
                if (ok != ok64 || (ok && bin != bin64)) diffs++;
            }
        }
    if (ndiff64) *ndiff64 = diffs;
    return votes;
}

/* Per-voxel decision for a list of global voxel indices (for analytic pins):
 * out[k] = bin, or -1 if no vote. */
void orc_vote_list(int64_t n, const int64_t* idx3, const double* origin, double h, double r,
                   const double* cam, int W, int H, const float* pyr, int nbins, int32_t* out)
{
    orc_cam32 c32 = orc_cam_from_f64(cam, W, H);
    int32_t dims[64];
    int64_t offs[32];
    int nlev = orc_pyramid_nlevels(W, H);
    orc_pyramid_layout(W, H, dims, offs);
    float o32[3] = {(float)origin[0], (float)origin[1], (float)origin[2]};
    for (int64_t k = 0; k < n; ++k) {
        int bin = -1;
        if (!orc_vote_f32(&c32, pyr, nlev, dims, offs, o32, (float)h, (float)r, idx3 + 3 * k, nbins, &bin))
            bin = -1;
        out[k] = bin;
    }
}

/* ======================================================================== */
/* Brick domain links.                                                      */
/* For each active voxel x and axis a: fwd(x,a), bwd(x,a) in                */
/*   ACT(y)  -> y >= 0 (active voxel id)                                    */
/*   NONE    -> -1     (outside the domain: Neumann, no difference)         */
/*   FRZ(k)  -> -2-k   (frozen voxel k = frozen_brick*512 + local; its u, v */
/*                      are constants: Sec. 4.5, set B keeps the parent's   */
/*                      indicator; reading: v is frozen too)                */
/* Returns 0, or -1 on a duplicate brick.                                   */
/* ======================================================================== */
typedef struct {
    int64_t key;
    int64_t id; /* >= 0 active brick; < 0: frozen brick -1-id */
} orc_bkey;

static int64_t orc_key(int64_t x, int64_t y, int64_t z)
{
    const int64_t B = 1 << 20;
    return ((z + B) * (2 * B) + (y + B)) * (2 * B) + (x + B);
}

static int orc_cmp(const void* a, const void* b)
{
    int64_t ka = ((const orc_bkey*)a)->key, kb = ((const orc_bkey*)b)->key;
    return ka < kb ? -1 : (ka > kb ? 1 : 0);
}

static int64_t orc_find(const orc_bkey* t, int64_t n, int64_t key)
{
    int64_t lo = 0, hi = n - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (t[mid].key == key) return mid;
        if (t[mid].key < key) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

int orc_build_links(int64_t nb, const int32_t* bricks, int64_t nf, const int32_t* frozen, int64_t* fwd,
                    int64_t* bwd)
{
    int64_t n = nb + nf;
    orc_bkey* t = (orc_bkey*)malloc(sizeof(orc_bkey) * (size_t)(n > 0 ? n : 1));
    for (int64_t b = 0; b < nb; ++b) {
        t[b].key = orc_key(bricks[3 * b], bricks[3 * b + 1], bricks[3 * b + 2]);
        t[b].id = b;
    }
    for (int64_t f = 0; f < nf; ++f) {
        t[nb + f].key = orc_key(frozen[3 * f], frozen[3 * f + 1], frozen[3 * f + 2]);
        t[nb + f].id = -1 - f;
    }
    qsort(t, (size_t)n, sizeof(orc_bkey), orc_cmp);
    for (int64_t k = 1; k < n; ++k)
        if (t[k].key == t[k - 1].key) {
            free(t);
            return -1;
        }
    for (int64_t b = 0; b < nb; ++b)
        for (int v = 0; v < ORC_BVOX; ++v) {
            int64_t g[3] = {(int64_t)ORC_BRICK * bricks[3 * b] + (v & 7),
                            (int64_t)ORC_BRICK * bricks[3 * b + 1] + ((v >> 3) & 7),
                            (int64_t)ORC_BRICK * bricks[3 * b + 2] + (v >> 6)};
            int64_t x = b * ORC_BVOX + v;
            for (int a = 0; a < 3; ++a)
                for (int s = 0; s < 2; ++s) {
                    int64_t q[3] = {g[0], g[1], g[2]};
                    q[a] += s == 0 ? 1 : -1;
                    /* floor division by 8 for negative coordinates */
                    int64_t bq[3], lq[3];
                    for (int c = 0; c < 3; ++c) {
                        bq[c] = q[c] >= 0 ? q[c] / ORC_BRICK : -((-q[c] + ORC_BRICK - 1) / ORC_BRICK);
                        lq[c] = q[c] - ORC_BRICK * bq[c];
                    }
                    int64_t pos = orc_find(t, n, orc_key(bq[0], bq[1], bq[2]));
                    int64_t link;
                    if (pos < 0) {
                        link = -1;
                    } else {
                        int64_t lv = lq[0] + 8 * lq[1] + 64 * lq[2];
                        if (t[pos].id >= 0) link = t[pos].id * ORC_BVOX + lv;
                        else link = -2 - ((-1 - t[pos].id) * ORC_BVOX + lv);
                    }
                    if (s == 0) fwd[3 * x + a] = link;
                    else bwd[3 * x + a] = link;
                }
        }
    free(t);
    return 0;
}

/* ======================================================================== */
/* TGV operators (Eq. 2-3), finite differences on the voxel grid with unit   */
/* index spacing (reading: spacing 1 on every level).                        */
/*   forward gradient       (grad u)_a(x) = u(fwd) - u(x), 0 if NONE          */
/*   backward difference    d-_a w(x)     = w(x) - w(bwd), 0 if NONE          */
/*   symmetric gradient     E(v)_ab = (d-_a v_b + d-_b v_a)/2   (Eq. 3)       */
/* FRZ neighbours contribute their frozen u / v.  The divergences below are  */
/* the exact negative adjoints of the linear parts (FRZ constants set to 0). */
/* q is stored as (q00, q11, q22, q01, q02, q12); Frobenius inner products   */
/* count the off-diagonal pair twice.                                        */
/* ======================================================================== */
static const int orc_qidx[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};

static double orc_u_at(int64_t link, const double* u, const double* fu)
{
    return link >= 0 ? u[link] : fu[-2 - link];
}

static void orc_grad_at(int64_t x, const int64_t* fwd, const double* u, const double* fu, double g[3])
{
    for (int a = 0; a < 3; ++a) {
        int64_t l = fwd[3 * x + a];
        g[a] = l == -1 ? 0.0 : orc_u_at(l, u, fu) - u[x];
    }
}

static void orc_symgrad_at(int64_t x, const int64_t* bwd, const double* v, const double* fv, double e[6])
{
    double dm[3][3]; /* dm[a][b] = d-_a v_b */
    for (int a = 0; a < 3; ++a) {
        int64_t l = bwd[3 * x + a];
        for (int b = 0; b < 3; ++b) {
            if (l == -1) dm[a][b] = 0.0;
            else if (l >= 0) dm[a][b] = v[3 * x + b] - v[3 * l + b];
            else dm[a][b] = v[3 * x + b] - fv[3 * (-2 - l) + b];
        }
    }
    e[0] = dm[0][0];
    e[1] = dm[1][1];
    e[2] = dm[2][2];
    e[3] = 0.5 * (dm[0][1] + dm[1][0]);
    e[4] = 0.5 * (dm[0][2] + dm[2][0]);
    e[5] = 0.5 * (dm[1][2] + dm[2][1]);
}

/* div1 p (x) = sum_a ( [fwd(x,a) != NONE] p_a(x) - [bwd(x,a) = ACT] p_a(bwd) ) */
static double orc_div1_at(int64_t x, const int64_t* fwd, const int64_t* bwd, const double* p)
{
    double s = 0.0;
    for (int a = 0; a < 3; ++a) {
        if (fwd[3 * x + a] != -1) s += p[3 * x + a];
        int64_t l = bwd[3 * x + a];
        if (l >= 0) s -= p[3 * l + a];
    }
    return s;
}

/* (div2 q)_b (x) = sum_a ( [fwd(x,a) = ACT] q_ab(fwd) - [bwd(x,a) != NONE] q_ab(x) ) */
static void orc_div2_at(int64_t x, const int64_t* fwd, const int64_t* bwd, const double* q, double w[3])
{
    for (int b = 0; b < 3; ++b) {
        double s = 0.0;
        for (int a = 0; a < 3; ++a) {
            int64_t lf = fwd[3 * x + a];
            if (lf >= 0) s += q[6 * lf + orc_qidx[a][b]];
            if (bwd[3 * x + a] != -1) s -= q[6 * x + orc_qidx[a][b]];
        }
        w[b] = s;
    }
}

/* Whole-field operator entry points (used by the adjoint / affine pins). */
void orc_grad(int64_t n, const int64_t* fwd, const double* u, const double* fu, double* g)
{
    for (int64_t x = 0; x < n; ++x) orc_grad_at(x, fwd, u, fu, g + 3 * x);
}
void orc_symgrad(int64_t n, const int64_t* bwd, const double* v, const double* fv, double* e)
{
    for (int64_t x = 0; x < n; ++x) orc_symgrad_at(x, bwd, v, fv, e + 6 * x);
}
void orc_div1(int64_t n, const int64_t* fwd, const int64_t* bwd, const double* p, double* d)
{
    for (int64_t x = 0; x < n; ++x) d[x] = orc_div1_at(x, fwd, bwd, p);
}
void orc_div2(int64_t n, const int64_t* fwd, const int64_t* bwd, const double* q, double* w)
{
    for (int64_t x = 0; x < n; ++x) orc_div2_at(x, fwd, bwd, q, w + 3 * x);
}

/* ======================================================================== */
/* Projections onto the dual constraint sets of Eq. 2:                       */
/*   |p|_2 <= alpha1,   |q|_F <= alpha0  (isotropic per voxel).              */
/* ======================================================================== */
static void orc_proj_p(double p[3], double alpha1)
{
    double n = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    double s = n / alpha1;
    if (s > 1.0)
        for (int a = 0; a < 3; ++a) p[a] /= s;
}

static void orc_proj_q(double q[6], double alpha0)
{
    double n2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + 2.0 * (q[3] * q[3] + q[4] * q[4] + q[5] * q[5]);
    double s = sqrt(n2) / alpha0;
    if (s > 1.0)
        for (int c = 0; c < 6; ++c) q[c] /= s;
}

void orc_project_p(int64_t n, double* p, double alpha1)
{
    for (int64_t x = 0; x < n; ++x) orc_proj_p(p + 3 * x, alpha1);
}
void orc_project_q(int64_t n, double* q, double alpha0)
{
    for (int64_t x = 0; x < n; ++x) orc_proj_q(q + 6 * x, alpha0);
}

/* ======================================================================== */
/* Histogram data term (Sec. 3.4, histograms after Zach 2008):               */
/*   sum_b h_b |u - c_b|,  bin centres c_b.                                  */
/* Reading: centres = 0 -> c_b = -1 + 2b/(n-1) (bin 0 = occluded -1, bin n-1 */
/*          = free space +1); centres = 1 -> interval midpoints              */
/*          c_b = -1 + (2b+1)/n.                                             */
/* Prox (generalised median): argmin_u (u-ut)^2/(2 tau) + lam sum h_b|u-c_b| */
/* = median of {c_0..c_{n-1}} U {ut - tau lam W_i, i = 0..n},                */
/*   W_i = sum_{b<i} h_b - sum_{b>=i} h_b.                                   */
/* ======================================================================== */
double orc_centre(int b, int n, int centres)
{
    return centres == 0 ? -1.0 + 2.0 * b / (double)(n - 1) : -1.0 + (2.0 * b + 1.0) / (double)n;
}

static int orc_dcmp(const void* a, const void* b)
{
    double x = *(const double*)a, y = *(const double*)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

double orc_prox(double ut, const uint32_t* hb, int n, double tau, double lam, int centres)
{
    double vals[2 * 64 + 1];
    int m = 0;
    for (int b = 0; b < n; ++b) vals[m++] = orc_centre(b, n, centres);
    for (int i = 0; i <= n; ++i) {
        double W = 0.0;
        for (int b = 0; b < n; ++b) W += b < i ? (double)hb[b] : -(double)hb[b];
        vals[m++] = ut - tau * lam * W;
    }
    qsort(vals, (size_t)m, sizeof(double), orc_dcmp);
    return vals[n]; /* the middle of 2n+1 sorted values */
}

/* Data term for one voxel. */
static double orc_data_at(double u, const uint32_t* hb, int n, double lam, int centres)
{
    double s = 0.0;
    for (int b = 0; b < n; ++b) s += (double)hb[b] * fabs(u - orc_centre(b, n, centres));
    return lam * s;
}

/* ======================================================================== */
/* One primal-dual iteration (Sec. 3.2: the primal-dual method of Pock et    */
/* al. 2011 for Eq. 2; reading: the Chambolle-Pock order below, theta = 1).  */
/*   1. p <- proj_alpha1(p + sigma (grad ubar - vbar))                       */
/*   2. q <- proj_alpha0(q + sigma E(vbar))                                  */
/*   3. ut <- u + tau div1 p                                                 */
/*   4. u+ <- clamp(prox(ut), -1, 1)   (clamp_u: indicator range, Sec. 3.2)  */
/*   5. v+ <- v + tau (p + div2 q)                                           */
/*   6. ubar <- 2u+ - u, vbar <- 2v+ - v;  u <- u+, v <- v+                  */
/* Steps 1-2 finish for every voxel before steps 3-6 start (Jacobi).         */
/* prm: alpha1, alpha0, lambda, tau, sigma.  Per-voxel loops are independent,*/
/* so the result does not depend on the thread count.                        */
/* ======================================================================== */
void orc_tgv_iterate(int64_t n, const int64_t* fwd, const int64_t* bwd, const double* fu, const double* fv,
                     const uint32_t* hist, int nbins, const double* prm, int clamp_u, int centres, double* u,
                     double* ubar, double* v, double* vbar, double* p, double* q, int iters, int nthreads)
{
    double alpha1 = prm[0], alpha0 = prm[1], lam = prm[2], tau = prm[3], sigma = prm[4];
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    double* pn = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double* qn = (double*)malloc(sizeof(double) * 6 * (size_t)(n > 0 ? n : 1));
    for (int it = 0; it < iters; ++it) {
#pragma omp parallel for schedule(static)
        for (int64_t x = 0; x < n; ++x) {
            double g[3], e[6];
            orc_grad_at(x, fwd, ubar, fu, g);
            for (int a = 0; a < 3; ++a) pn[3 * x + a] = p[3 * x + a] + sigma * (g[a] - vbar[3 * x + a]);
            orc_proj_p(pn + 3 * x, alpha1);
            orc_symgrad_at(x, bwd, vbar, fv, e);
            for (int c = 0; c < 6; ++c) qn[6 * x + c] = q[6 * x + c] + sigma * e[c];
            orc_proj_q(qn + 6 * x, alpha0);
        }
        memcpy(p, pn, sizeof(double) * 3 * (size_t)n);
        memcpy(q, qn, sizeof(double) * 6 * (size_t)n);
#pragma omp parallel for schedule(static)
        for (int64_t x = 0; x < n; ++x) {
            double ut = u[x] + tau * orc_div1_at(x, fwd, bwd, p);
            double un = orc_prox(ut, hist + x * nbins, nbins, tau, lam, centres);
            if (clamp_u) un = un < -1.0 ? -1.0 : (un > 1.0 ? 1.0 : un);
            double w[3];
            orc_div2_at(x, fwd, bwd, q, w);
            for (int a = 0; a < 3; ++a) {
                double vn = v[3 * x + a] + tau * (p[3 * x + a] + w[a]);
                vbar[3 * x + a] = 2.0 * vn - v[3 * x + a];
                v[3 * x + a] = vn;
            }
            ubar[x] = 2.0 * un - u[x];
            u[x] = un;
        }
    }
    free(pn);
    free(qn);
}

/* ======================================================================== */
/* Energy of Eq. 2 on the discrete domain, dual value and gap.              */
/*   E(u,v) = alpha1 sum |grad u - v|_2 + alpha0 sum |E v|_F                */
/*            + lam sum_x sum_b h_b |u - c_b|         (FRZ constants in)    */
/* Reading (bounded primal sets so the gap is finite): u in [-1, 1] and    */
/* every component |v_a| <= Bv.  With K(u,v) = K0(u,v) + k0 (k0 = the FRZ    */
/* constants, i.e. K(0,0)):                                                 */
/*   D(p,q) = <k0,(p,q)> - sum_x phi*_x(div1 p(x)) - Bv |p + div2 q|_1       */
/*   phi*_x(w) = max over u in {-1, c_0..c_{n-1}, +1} of                     */
/*               w u - lam sum_b h_b |u - c_b|    (concave piecewise linear) */
/* out[0] = E, out[1] = D, out[2] = E - D, out[3] = 1 if every |v_a| <= Bv.  */
/* Sums run serially in voxel order.                                        */
/* ======================================================================== */
void orc_energy(int64_t n, const int64_t* fwd, const int64_t* bwd, const double* fu, const double* fv,
                const uint32_t* hist, int nbins, const double* prm, int centres, double Bv, const double* u,
                const double* v, const double* p, const double* q, double* out)
{
    double alpha1 = prm[0], alpha0 = prm[1], lam = prm[2];
    double E = 0.0, D = 0.0;
    int certified = 1;
    double* zeros_u = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double* zeros_v = (double*)calloc(3 * (size_t)(n > 0 ? n : 1), sizeof(double));
    for (int64_t x = 0; x < n; ++x) {
        double g[3], e[6], w[3];
        /* primal */
        orc_grad_at(x, fwd, u, fu, g);
        double s = 0.0;
        for (int a = 0; a < 3; ++a) {
            double t = g[a] - v[3 * x + a];
            s += t * t;
            if (fabs(v[3 * x + a]) > Bv) certified = 0;
        }
        E += alpha1 * sqrt(s);
        orc_symgrad_at(x, bwd, v, fv, e);
        double f2 = e[0] * e[0] + e[1] * e[1] + e[2] * e[2] + 2.0 * (e[3] * e[3] + e[4] * e[4] + e[5] * e[5]);
        E += alpha0 * sqrt(f2);
        E += orc_data_at(u[x], hist + x * nbins, nbins, lam, centres);
        /* dual: <k0, (p, q)> */
        orc_grad_at(x, fwd, zeros_u, fu, g);
        orc_symgrad_at(x, bwd, zeros_v, fv, e);
        double k = 0.0;
        for (int a = 0; a < 3; ++a) k += g[a] * p[3 * x + a];
        k += e[0] * q[6 * x] + e[1] * q[6 * x + 1] + e[2] * q[6 * x + 2] +
             2.0 * (e[3] * q[6 * x + 3] + e[4] * q[6 * x + 4] + e[5] * q[6 * x + 5]);
        D += k;
        /* dual: - phi*(div1 p) */
        double dv = orc_div1_at(x, fwd, bwd, p);
        double best = -INFINITY;
        for (int c = -1; c <= nbins; ++c) {
            double uu = c < 0 ? -1.0 : (c == nbins ? 1.0 : orc_centre(c, nbins, centres));
            double val = dv * uu - orc_data_at(uu, hist + x * nbins, nbins, lam, centres);
            if (val > best) best = val;
        }
        D -= best;
        /* dual: - Bv |p + div2 q|_1 */
        orc_div2_at(x, fwd, bwd, q, w);
        for (int a = 0; a < 3; ++a) D -= Bv * fabs(p[3 * x + a] + w[a]);
    }
    free(zeros_u);
    free(zeros_v);
    out[0] = E;
    out[1] = D;
    out[2] = E - D;
    out[3] = certified ? 1.0 : 0.0;
}

/* ======================================================================== */
/* Coarse-to-fine initialisation (Sec. 4.5; reading: piecewise-constant     */
/* prolongation of u, v halved because the index spacing halves, duals      */
/* restart at zero).  Level l+1 shares the origin of level l and has half   */
/* its voxel edge, so fine voxel g has parent floor(g/2).                   */
/* fine_vox3: (nf, 3) global fine voxel indices; parent lookup by the       */
/* coarse brick list.  Missing parents leave u = v = 0 and are counted.     */
/* ======================================================================== */
int64_t orc_prolong(int64_t nbc, const int32_t* cbricks, const double* cu, const double* cv, int64_t nfv,
                    const int64_t* fine_vox3, double* fu, double* fv)
{
    orc_bkey* t = (orc_bkey*)malloc(sizeof(orc_bkey) * (size_t)(nbc > 0 ? nbc : 1));
    for (int64_t b = 0; b < nbc; ++b) {
        t[b].key = orc_key(cbricks[3 * b], cbricks[3 * b + 1], cbricks[3 * b + 2]);
        t[b].id = b;
    }
    qsort(t, (size_t)nbc, sizeof(orc_bkey), orc_cmp);
    int64_t missing = 0;
    for (int64_t k = 0; k < nfv; ++k) {
        int64_t c[3], bq[3], lq[3];
        for (int a = 0; a < 3; ++a) {
            int64_t g = fine_vox3[3 * k + a];
            c[a] = g >= 0 ? g / 2 : -((-g + 1) / 2);
            bq[a] = c[a] >= 0 ? c[a] / ORC_BRICK : -((-c[a] + ORC_BRICK - 1) / ORC_BRICK);
            lq[a] = c[a] - ORC_BRICK * bq[a];
        }
        int64_t pos = orc_find(t, nbc, orc_key(bq[0], bq[1], bq[2]));
        if (pos < 0) {
            fu[k] = 0.0;
            for (int a = 0; a < 3; ++a) fv[3 * k + a] = 0.0;
            missing++;
            continue;
        }
        int64_t cx = t[pos].id * ORC_BVOX + lq[0] + 8 * lq[1] + 64 * lq[2];
        fu[k] = cu[cx];
        for (int a = 0; a < 3; ++a) fv[3 * k + a] = 0.5 * cv[3 * cx + a];
    }
    free(t);
    return missing;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ======================================================================== */
/* Marching cubes on a brick level (Sec. 4.6): for every cube whose corners   */
/* take indicator values of different sign, the points where u crosses zero  */
/* along its edges, joined into closed polygons and triangulated by dynamic  */
/* programming that minimises the total area (after Bloomenthal 1988).       */
/*                                                                          */
/* Readings (the paper gives no more detail):                                */
/*  - a cube ("cell") has 8 voxel centres as corners; the cell with lower    */
/*    corner voxel g is extracted when g lies in an active brick and all 8   */
/*    corners exist (active or frozen bricks);                               */
/*  - corner c = dx + 2 dy + 4 dz is inside when u < 0 (u = -1 interior);    */
/*  - an edge from voxel p to p + e_a crosses when exactly one end is inside; */
/*    its point is at t = u_p / (u_p - u_q) along the edge; coordinates      */
/*    o + ((g + 0.5) + t) h on axis a, o + (g + 0.5) h on the others, all in */
/*    FP32 with one rounding per operation;                                  */
/*  - each face of the cell, corners counter-clockwise seen from outside the */
/*    cell, joins a crossing where the boundary enters the inside region to  */
/*    the next crossing where it leaves; on a face with four crossings the   */
/*    face sum ((u_a + u_b) + (u_c + u_d)) over its corners in cell order    */
/*    decides: >= 0 joins each entry to the next exit (inside corners apart),*/
/*    < 0 to the previous exit (inside corners connected).  The two cells    */
/*    sharing a face see the same corners in the same order and decide alike;*/
/*  - segments run entry -> exit, so every polygon is counter-clockwise seen */
/*    from the outside region (u >= 0) and triangle normals point there;     */
/*  - a polygon P0..P(k-1) (P0 = its crossing on the cell edge of lowest     */
/*    index 4a + (other two corner bits)) is triangulated by                 */
/*      C[i][j] = min_{i<m<j} (C[i][m] + C[m][j]) + |(Pm - Pi) x (Pj - Pi)|  */
/*    in FP32 (ties: smallest m), triangles emitted root first, then the     */
/*    (i, m) side, then the (m, j) side, each as (Pi, Pm, Pj);               */
/*  - a polygon with no triangulation free of chords along a cell face (one */
/*    that carries the segments of several four-crossing faces) is fanned    */
/*    around its centroid (FP32 sum in polygon order, divided by k), a vertex */
/*    of the cell; at most one per cell, later ones take the unconstrained   */
/*    triangulation;                                                         */
/*  - vertices are numbered by increasing id: 4 slot(p) + a for the crossing */
/*    on the edge from voxel p along axis a, 4 slot(g) + 3 for the centroid  */
/*    of the cell with lower corner g; slot = brick * 512 + local and frozen */
/*    brick f has brick index nb + f;                                        */
/*    triangles come in increasing cell order (active brick, local index).   */
/* ======================================================================== */
#define ORC_MC_MAXV 12

static const int orc_mc_face[6][4] = {{0, 4, 6, 2}, {1, 3, 7, 5}, {0, 1, 5, 4},
                                      {2, 6, 7, 3}, {0, 2, 3, 1}, {4, 5, 7, 6}};

/* cell edge index of the edge between corners c0 and c1 (they differ in one bit) */
static int orc_mc_edge(int c0, int c1)
{
    int lo = c0 < c1 ? c0 : c1, x = c0 ^ c1;
    int a = x == 1 ? 0 : (x == 2 ? 1 : 2);
    int bits[3] = {lo & 1, (lo >> 1) & 1, (lo >> 2) & 1};
    int m = 0, s = 0;
    for (int b = 0; b < 3; ++b)
        if (b != a) m |= bits[b] << s++;
    return 4 * a + m;
}

/* base corner and axis of cell edge e */
static void orc_mc_edge_base(int e, int* base, int* axis)
{
    int a = e / 4, m = e % 4, bits[3] = {0, 0, 0}, s = 0;
    for (int b = 0; b < 3; ++b)
        if (b != a) bits[b] = (m >> s++) & 1;
    *base = bits[0] + 2 * bits[1] + 4 * bits[2];
    *axis = a;
}

static float orc_mc_area2(const float* P, int i, int m, int j)
{
    float e1[3], e2[3];
    for (int c = 0; c < 3; ++c) {
        e1[c] = P[3 * m + c] - P[3 * i + c];
        e2[c] = P[3 * j + c] - P[3 * i + c];
    }
    float cx = e1[1] * e2[2] - e1[2] * e2[1];
    float cy = e1[2] * e2[0] - e1[0] * e2[2];
    float cz = e1[0] * e2[1] - e1[1] * e2[0];
    float n2 = cx * cx + cy * cy;
    n2 = n2 + cz * cz;
    return sqrtf(n2);
}

/* 1 when cell edges e1 and e2 lie on a common face of the cell: a face fixes
 * one coordinate bit f, and an edge of axis a with base corner b lies on the
 * faces f != a with bit f of b as the fixed value. */
static int orc_mc_share_face(int e1, int e2)
{
    int b1, a1, b2, a2;
    orc_mc_edge_base(e1, &b1, &a1);
    orc_mc_edge_base(e2, &b2, &a2);
    for (int f = 0; f < 3; ++f)
        if (f != a1 && f != a2 && ((b1 >> f) & 1) == ((b2 >> f) & 1)) return 1;
    return 0;
}

/* Minimum-area triangulation of the polygon P[0..k-1] (3 floats per vertex) by
 * dynamic programming over chords, FP32 with the operation order of
 * orc_mc_area2: C[i][j] = min_{i<m<j} (C[i][m] + C[m][j]) + area2(i, m, j),
 * ties to the smallest m; triangles (i, m, j) emitted root first, then the
 * (i, m) side, then the (m, j) side.  Returns the number of triangles (k - 2).
 * cell_edges (nullable): the cell edge of each vertex; a chord between two
 * vertices on a common cell face is then not allowed (the neighbouring cell
 * would place the opposite triangle in that face); returns -1 when every
 * triangulation needs one. */
int orc_mc_triangulate(int k, const float* P, const int* cell_edges, int* tri)
{
    float C[ORC_MC_MAXV][ORC_MC_MAXV];
    int best[ORC_MC_MAXV][ORC_MC_MAXV];
    if (k < 3 || k > ORC_MC_MAXV) return 0;
    {
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j) {
                C[i][j] = 0.0f;
                best[i][j] = j == i + 1 ? k : -1; /* polygon edges: valid, no triangle */
            }
        for (int len = 2; len < k; ++len)
            for (int i = 0; i + len < k; ++i) {
                int j = i + len;
                if (cell_edges && len < k - 1 && orc_mc_share_face(cell_edges[i], cell_edges[j])) continue;
                float bc = 0.0f;
                int bm = -1;
                for (int m = i + 1; m < j; ++m) {
                    if (best[i][m] < 0 || best[m][j] < 0) continue;
                    float c = (C[i][m] + C[m][j]) + orc_mc_area2(P, i, m, j);
                    if (bm < 0 || c < bc) {
                        bc = c;
                        bm = m;
                    }
                }
                C[i][j] = bc;
                best[i][j] = bm;
            }
        if (best[0][k - 1] < 0) return -1;
    }
    int st[2 * ORC_MC_MAXV][2], sp = 0, nt = 0;
    st[sp][0] = 0;
    st[sp][1] = k - 1;
    sp++;
    while (sp > 0) {
        sp--;
        int i = st[sp][0], j = st[sp][1];
        if (j - i < 2) continue;
        int m = best[i][j];
        tri[3 * nt + 0] = i;
        tri[3 * nt + 1] = m;
        tri[3 * nt + 2] = j;
        nt++;
        st[sp][0] = m; /* (m, j) below (i, m): (i, m) comes out first */
        st[sp][1] = j;
        sp++;
        st[sp][0] = i;
        st[sp][1] = m;
        sp++;
    }
    return nt;
}

typedef struct {
    const orc_bkey* t;
    int64_t nall, nb;
    const int32_t* bricks;
    const int32_t* frozen;
    const float* u;
    float o[3], h;
} orc_mc_ctx;

/* slot of the voxel at global coordinates g, or -1 */
static int64_t orc_mc_slot(const orc_mc_ctx* X, const int64_t g[3])
{
    int64_t bq[3], lq[3];
    for (int c = 0; c < 3; ++c) {
        bq[c] = g[c] >= 0 ? g[c] / ORC_BRICK : -((-g[c] + ORC_BRICK - 1) / ORC_BRICK);
        lq[c] = g[c] - ORC_BRICK * bq[c];
    }
    int64_t pos = orc_find(X->t, X->nall, orc_key(bq[0], bq[1], bq[2]));
    if (pos < 0) return -1;
    int64_t id = X->t[pos].id, brick = id >= 0 ? id : X->nb + (-1 - id);
    return brick * ORC_BVOX + lq[0] + 8 * lq[1] + 64 * lq[2];
}

static void orc_mc_slot_coords(const orc_mc_ctx* X, int64_t slot, int64_t g[3])
{
    int64_t b = slot / ORC_BVOX, v = slot % ORC_BVOX;
    const int32_t* bc = b < X->nb ? X->bricks + 3 * b : X->frozen + 3 * (b - X->nb);
    g[0] = (int64_t)ORC_BRICK * bc[0] + (v & 7);
    g[1] = (int64_t)ORC_BRICK * bc[1] + ((v >> 3) & 7);
    g[2] = (int64_t)ORC_BRICK * bc[2] + (v >> 6);
}

/* FP32 position of the zero crossing on edge id = 4 slot + axis (axis < 3) */
static void orc_mc_vertex(const orc_mc_ctx* X, int64_t eid, float out[3])
{
    int64_t slot = eid / 4, g[3], gq[3];
    int a = (int)(eid % 4);
    orc_mc_slot_coords(X, slot, g);
    for (int c = 0; c < 3; ++c) gq[c] = g[c] + (c == a);
    float up = X->u[slot], uq = X->u[orc_mc_slot(X, gq)];
    float t = up / (up - uq);
    for (int c = 0; c < 3; ++c) {
        float s = (float)g[c] + 0.5f;
        if (c == a) s = s + t;
        out[c] = X->o[c] + s * X->h;
    }
}

typedef struct {
    int64_t id;
    float p[3];
} orc_mc_centre;

static int orc_mc_cmp64(const void* a, const void* b)
{
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

static int64_t orc_mc_rank(const int64_t* ids, int64_t n, int64_t id)
{
    int64_t lo = 0, hi = n - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (ids[mid] == id) return mid;
        if (ids[mid] < id) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

/* One cell: its global edge ids of crossed edges (eid[12], -1 if not crossed),
 * its polygons (loop vertex lists as cell edges) and the triangles of each.
 * Returns the number of triangles, writes them as cell edge triples. */
static int orc_mc_cell(const orc_mc_ctx* X, const int64_t g0[3], int64_t eid[13], int tri[ORC_MC_MAXV * 3],
                       float centre[3], int* centre_used)
{
    *centre_used = 0;
    int64_t slot[8];
    float uc[8];
    for (int c = 0; c < 8; ++c) {
        int64_t g[3] = {g0[0] + (c & 1), g0[1] + ((c >> 1) & 1), g0[2] + (c >> 2)};
        slot[c] = orc_mc_slot(X, g);
        if (slot[c] < 0) return -1;
        uc[c] = X->u[slot[c]];
    }
    int inside[8], any_in = 0, any_out = 0;
    for (int c = 0; c < 8; ++c) {
        inside[c] = uc[c] < 0.0f;
        any_in |= inside[c];
        any_out |= !inside[c];
    }
    for (int e = 0; e < 13; ++e) eid[e] = -1;
    if (!any_in || !any_out) return 0;
    for (int e = 0; e < 12; ++e) {
        int base, a;
        orc_mc_edge_base(e, &base, &a);
        if (inside[base] != inside[base | (1 << a)]) eid[e] = 4 * slot[base] + a;
    }
    eid[12] = 4 * slot[0] + 3; /* the cell's centre vertex, used only by a fan */
    /* next[e]: the segment starting at crossing e (where it is an entry) ends at next[e] */
    int next[12];
    for (int e = 0; e < 12; ++e) next[e] = -1;
    for (int f = 0; f < 6; ++f) {
        const int* k = orc_mc_face[f];
        int ne = 0, pos_e[4], typ[4];
        for (int m = 0; m < 4; ++m) {
            int c0 = k[m], c1 = k[(m + 1) % 4];
            typ[m] = inside[c0] == inside[c1] ? 0 : (inside[c0] ? 2 /* exit */ : 1 /* entry */);
            pos_e[m] = orc_mc_edge(c0, c1);
        }
        for (int m = 0; m < 4; ++m) ne += typ[m] != 0;
        if (ne == 0) continue;
        int connected_inside = 0;
        if (ne == 4) {
            int s[4] = {k[0], k[1], k[2], k[3]};
            /* corners in cell order */
            for (int x = 0; x < 4; ++x)
                for (int y = x + 1; y < 4; ++y)
                    if (s[y] < s[x]) {
                        int tmp = s[x];
                        s[x] = s[y];
                        s[y] = tmp;
                    }
            float sum = (uc[s[0]] + uc[s[1]]) + (uc[s[2]] + uc[s[3]]);
            connected_inside = sum < 0.0f;
        }
        for (int m = 0; m < 4; ++m) {
            if (typ[m] != 1) continue;
            int p = -1;
            if (!connected_inside) {
                for (int d = 1; d < 4; ++d)
                    if (typ[(m + d) % 4] == 2) {
                        p = (m + d) % 4;
                        break;
                    }
            } else {
                for (int d = 1; d < 4; ++d)
                    if (typ[(m + 4 - d) % 4] == 2) {
                        p = (m + 4 - d) % 4;
                        break;
                    }
            }
            next[pos_e[m]] = pos_e[p];
        }
    }
    int ntri = 0, done[12] = {0};
    for (int e0 = 0; e0 < 12; ++e0) {
        if (eid[e0] < 0 || done[e0]) continue;
        int poly[ORC_MC_MAXV], k = 0, e = e0;
        do {
            poly[k++] = e;
            done[e] = 1;
            e = next[e];
        } while (e != e0 && e >= 0 && k < ORC_MC_MAXV);
        float P[3 * ORC_MC_MAXV];
        for (int v = 0; v < k; ++v) orc_mc_vertex(X, eid[poly[v]], P + 3 * v);
        int lt[3 * ORC_MC_MAXV];
        int nt = orc_mc_triangulate(k, P, poly, lt);
        if (nt < 0 && !*centre_used) {
            /* fan around the polygon's centroid (vertex 12 of the cell) */
            float c[3] = {0.0f, 0.0f, 0.0f};
            for (int v = 0; v < k; ++v)
                for (int q = 0; q < 3; ++q) c[q] = c[q] + P[3 * v + q];
            for (int q = 0; q < 3; ++q) centre[q] = c[q] / (float)k;
            *centre_used = 1;
            for (int v = 0; v < k; ++v) {
                tri[3 * ntri + 0] = poly[v];
                tri[3 * ntri + 1] = poly[(v + 1) % k];
                tri[3 * ntri + 2] = 12;
                ntri++;
            }
            continue;
        }
        if (nt < 0) nt = orc_mc_triangulate(k, P, NULL, lt);
        for (int q = 0; q < 3 * nt; ++q) tri[3 * ntri + q] = poly[lt[q]];
        ntri += nt;
    }
    return ntri;
}

/*
 * u: FP32 indicator of (nb + nf) * 512 voxels (active bricks, then frozen).
 * First call with verts = tris = NULL: returns the triangle count and sets
 * *nverts.  Second call with buffers of 3 * nverts floats and 3 * ntris int32
 * fills them.  Returns -1 on a duplicate brick.
 */
int64_t orc_mesh(int64_t nb, const int32_t* bricks, int64_t nf, const int32_t* frozen, const float* u,
                 const double* origin, double h, int64_t* nverts, float* verts, int32_t* tris)
{
    int64_t nall = nb + nf;
    orc_bkey* t = (orc_bkey*)malloc(sizeof(orc_bkey) * (size_t)(nall > 0 ? nall : 1));
    for (int64_t b = 0; b < nb; ++b) {
        t[b].key = orc_key(bricks[3 * b], bricks[3 * b + 1], bricks[3 * b + 2]);
        t[b].id = b;
    }
    for (int64_t f = 0; f < nf; ++f) {
        t[nb + f].key = orc_key(frozen[3 * f], frozen[3 * f + 1], frozen[3 * f + 2]);
        t[nb + f].id = -1 - f;
    }
    qsort(t, (size_t)nall, sizeof(orc_bkey), orc_cmp);
    for (int64_t k = 1; k < nall; ++k)
        if (t[k].key == t[k - 1].key) {
            free(t);
            return -1;
        }
    orc_mc_ctx X = {t, nall, nb, bricks, frozen, u, {(float)origin[0], (float)origin[1], (float)origin[2]}, (float)h};
    /* pass 1: referenced edges and cell centres */
    int64_t cap = 1024, ne = 0, ntri = 0, capc = 16, nc = 0;
    int64_t* ids = (int64_t*)malloc(sizeof(int64_t) * (size_t)cap);
    orc_mc_centre* cen = (orc_mc_centre*)malloc(sizeof(orc_mc_centre) * (size_t)capc);
    for (int64_t b = 0; b < nb; ++b)
        for (int v = 0; v < ORC_BVOX; ++v) {
            int64_t g0[3] = {(int64_t)ORC_BRICK * bricks[3 * b] + (v & 7), (int64_t)ORC_BRICK * bricks[3 * b + 1] + ((v >> 3) & 7),
                             (int64_t)ORC_BRICK * bricks[3 * b + 2] + (v >> 6)};
            int64_t eid[13];
            int tri[3 * ORC_MC_MAXV], cu;
            float cp[3];
            int n = orc_mc_cell(&X, g0, eid, tri, cp, &cu);
            if (n <= 0) continue;
            ntri += n;
            for (int e = 0; e < 13; ++e)
                if (eid[e] >= 0 && (e < 12 || cu)) {
                    if (ne == cap) {
                        cap *= 2;
                        ids = (int64_t*)realloc(ids, sizeof(int64_t) * (size_t)cap);
                    }
                    ids[ne++] = eid[e];
                }
            if (cu) {
                if (nc == capc) {
                    capc *= 2;
                    cen = (orc_mc_centre*)realloc(cen, sizeof(orc_mc_centre) * (size_t)capc);
                }
                cen[nc].id = eid[12];
                for (int q = 0; q < 3; ++q) cen[nc].p[q] = cp[q];
                nc++;
            }
        }
    qsort(ids, (size_t)ne, sizeof(int64_t), orc_mc_cmp64);
    int64_t nu = 0;
    for (int64_t k = 0; k < ne; ++k)
        if (k == 0 || ids[k] != ids[k - 1]) ids[nu++] = ids[k];
    *nverts = nu;
    if (verts)
        for (int64_t k = 0; k < nu; ++k) {
            if (ids[k] % 4 != 3) {
                orc_mc_vertex(&X, ids[k], verts + 3 * k);
                continue;
            }
            for (int64_t c = 0; c < nc; ++c)
                if (cen[c].id == ids[k])
                    for (int q = 0; q < 3; ++q) verts[3 * k + q] = cen[c].p[q];
        }
    if (tris) {
        int64_t o = 0;
        for (int64_t b = 0; b < nb; ++b)
            for (int v = 0; v < ORC_BVOX; ++v) {
                int64_t g0[3] = {(int64_t)ORC_BRICK * bricks[3 * b] + (v & 7),
                                 (int64_t)ORC_BRICK * bricks[3 * b + 1] + ((v >> 3) & 7),
                                 (int64_t)ORC_BRICK * bricks[3 * b + 2] + (v >> 6)};
                int64_t eid[13];
                int tri[3 * ORC_MC_MAXV], cu;
                float cp[3];
                int n = orc_mc_cell(&X, g0, eid, tri, cp, &cu);
                for (int k = 0; k < 3 * n; ++k) tris[o++] = (int32_t)orc_mc_rank(ids, nu, eid[tri[k]]);
            }
    }
    free(cen);
    free(ids);
    free(t);
    return ntri;
}

/* ======================================================================== */
/* Octree domain from depth maps (Sec. 3.3 Eq. 4, Sec. 4.1-4.3), in memory.  */
/*                                                                          */
/* Readings (the paper's out-of-core files become arrays):                   */
/*  - root cube [m, m + E)^3, radius r_root = E / 2;                         */
/*  - sample of pixel (i, j) with valid z-depth z (pinhole map):             */
/*      Pc = (((i + 0.5) - cx) / fx * z, ((j + 0.5) - cy) / fy * z, z)       */
/*      X_a = C_a + ((R0a Pc0 + R1a Pc1) + R2a Pc2)    (R rows = camera axes) */
/*    radius r = 0.5 * (sum of |X - X_n| over the valid 4-neighbours n, in   */
/*    the order left, right, up, down) / their count; none valid: no sample;  */
/*  - depth d (Eq. 4): the smallest d in [dmin, dmax] with                    */
/*    r_root * 2^-d < 1.5 r (so 0.75 r <= r_root 2^-d above dmin), else dmax;*/
/*  - cube q_a = floor(((X_a - m_a) / E) * 2^d), dropped outside [0, 2^d);    */
/*  - all of it in FP32, one rounding per operation, parameters rounded once;*/
/*  - level l = d - dmin has voxel edge E / 2^d, origin m; its bricks are the */
/*    cubes' q >> 3, dilated `band` times by their 26 neighbours (inside the */
/*    root); then, finest first, level l-1 gains the parents (b >> 1) of      */
/*    level l's bricks, dilated once (2:1 balance: a finer level is wrapped  */
/*    by a shell of the next coarser one);                                   */
/*  - frozen bricks of level l > 0: the 26-neighbours of its active bricks   */
/*    that are not active (inside the root);                                 */
/*  - bricks of a level are listed in Morton (Z-curve) order of their coords.*/
/* ======================================================================== */
static uint64_t orc_spread3(uint64_t v)
{
    uint64_t r = 0;
    for (int b = 0; b < 21; ++b) r |= ((v >> b) & 1u) << (3 * b);
    return r;
}

static uint64_t orc_morton(int64_t x, int64_t y, int64_t z)
{
    return orc_spread3((uint64_t)x) | (orc_spread3((uint64_t)y) << 1) | (orc_spread3((uint64_t)z) << 2);
}

/* sin and cos of x in FP32 (|x| <= 4), one rounding per operation: Cody-Waite
 * reduction by pi/2 -- k = nearest integer to x (2/pi), r = x - k pi/2 in two fused
 * multiply-adds with pi/2 split into a float head and tail -- then the Taylor
 * polynomials of sin (to r^9) and cos (to r^10) on |r| <= pi/4 (truncation below
 * 2e-9) by Horner's rule in fused multiply-adds, and the quadrant k mod 4. */
void orc_sincos_tay(float x, float* s, float* c)
{
    const float two_over_pi = (float)(2.0 / 3.14159265358979323846);
    const float p1 = (float)(3.14159265358979323846 / 2.0);
    const float p2 = (float)(3.14159265358979323846 / 2.0 - (double)p1);
    const float kf = rintf(x * two_over_pi);
    float r = fmaf(-kf, p1, x);
    r = fmaf(-kf, p2, r);
    const float r2 = r * r;
    float ps = fmaf(r2, (float)(1.0 / 362880.0), (float)(-1.0 / 5040.0));
    ps = fmaf(ps, r2, (float)(1.0 / 120.0));
    ps = fmaf(ps, r2, (float)(-1.0 / 6.0));
    const float sr = fmaf(r2 * r, ps, r);
    float pc = fmaf(r2, (float)(-1.0 / 3628800.0), (float)(1.0 / 40320.0));
    pc = fmaf(pc, r2, (float)(-1.0 / 720.0));
    pc = fmaf(pc, r2, (float)(1.0 / 24.0));
    pc = fmaf(pc, r2, -0.5f);
    const float cr = fmaf(pc, r2, 1.0f);
    switch ((int)kf & 3) {
    case 0: *s = sr; *c = cr; break;
    case 1: *s = cr; *c = -sr; break;
    case 2: *s = -sr; *c = -cr; break;
    default: *s = -cr; *c = sr; break;
    }
}

void orc_sincos_tay_many(const float* x, int64_t n, float* s, float* c)
{
    for (int64_t i = 0; i < n; ++i) orc_sincos_tay(x[i], s + i, c + i);
}

/* One sample per valid pixel of one map: writes depth d (or -1) and cube coords.
 * Pinhole: the camera-frame point ((i + 0.5 - cx) / fx z, (j + 0.5 - cy) / fy z, z).
 * Spherical (a LIDAR scan, z = range): azimuth phi = (i + 0.5 - cx) / fx, elevation
 * theta = (cy - (j + 0.5)) / fy, point z (cos theta cos phi, cos theta sin phi,
 * sin theta) with orc_sincos_tay. */
int64_t orc_octree_samples(const double* cam, int W, int H, const float* depth, const double* root_min, double root_edge,
                           int dmin, int dmax, int32_t* d_out, int64_t* q_out, float* r_out)
{
    float fx = (float)cam[0], fy = (float)cam[1], cx = (float)cam[2], cy = (float)cam[3];
    float R[9], C[3], m[3];
    for (int k = 0; k < 9; ++k) R[k] = (float)cam[4 + k];
    for (int k = 0; k < 3; ++k) C[k] = (float)cam[13 + k];
    for (int k = 0; k < 3; ++k) m[k] = (float)root_min[k];
    float E = (float)root_edge, rroot = E * 0.5f;
    const int spherical = cam[16] == 1.0;
    float* X = (float*)malloc(sizeof(float) * 3 * (size_t)W * (size_t)H);
    char* ok = (char*)malloc((size_t)W * (size_t)H);
    for (int j = 0; j < H; ++j)
        for (int i = 0; i < W; ++i) {
            int64_t p = (int64_t)j * W + i;
            float z = depth[p];
            ok[p] = isfinite(z) && z > 0.0f;
            if (!ok[p]) continue;
            float pc[3];
            if (spherical) {
                float sp, cp, st, ct;
                orc_sincos_tay((((float)i + 0.5f) - cx) / fx, &sp, &cp);
                orc_sincos_tay((cy - ((float)j + 0.5f)) / fy, &st, &ct);
                const float rc = z * ct;
                pc[0] = rc * cp;
                pc[1] = rc * sp;
                pc[2] = z * st;
            } else {
                pc[0] = (((float)i + 0.5f) - cx) / fx * z;
                pc[1] = (((float)j + 0.5f) - cy) / fy * z;
                pc[2] = z;
            }
            for (int a = 0; a < 3; ++a) {
                float s = R[0 + a] * pc[0] + R[3 + a] * pc[1];
                s = s + R[6 + a] * pc[2];
                X[3 * p + a] = C[a] + s;
            }
        }
    int64_t n = 0;
    for (int j = 0; j < H; ++j)
        for (int i = 0; i < W; ++i) {
            int64_t p = (int64_t)j * W + i;
            d_out[p] = -1;
            if (!ok[p]) continue;
            const int di[4] = {-1, 1, 0, 0}, dj[4] = {0, 0, -1, 1};
            float sum = 0.0f;
            int cnt = 0;
            for (int k = 0; k < 4; ++k) {
                int ii = i + di[k], jj = j + dj[k];
                if (ii < 0 || ii >= W || jj < 0 || jj >= H) continue;
                int64_t q = (int64_t)jj * W + ii;
                if (!ok[q]) continue;
                float e0 = X[3 * q] - X[3 * p], e1 = X[3 * q + 1] - X[3 * p + 1], e2 = X[3 * q + 2] - X[3 * p + 2];
                float l2 = e0 * e0 + e1 * e1;
                l2 = l2 + e2 * e2;
                sum = sum + sqrtf(l2);
                cnt++;
            }
            if (cnt == 0) continue;
            float r = 0.5f * (sum / (float)cnt);
            int d = dmin;
            while (d < dmax && !(ldexpf(rroot, -d) < 1.5f * r)) d++;
            int64_t q3[3];
            int inside = 1;
            for (int a = 0; a < 3; ++a) {
                float s = (X[3 * p + a] - m[a]) / E;
                float t = ldexpf(s, d);
                if (!(t >= 0.0f && t < ldexpf(1.0f, d))) inside = 0;
                q3[a] = inside ? (int64_t)floorf(t) : 0;
            }
            if (!inside) continue;
            d_out[p] = d;
            for (int a = 0; a < 3; ++a) q_out[3 * p + a] = q3[a];
            if (r_out) r_out[p] = r;
            n++;
        }
    free(X);
    free(ok);
    return n;
}

typedef struct {
    uint64_t key;
    int64_t c[3];
} orc_obrick;

static int orc_obrick_cmp(const void* a, const void* b)
{
    uint64_t x = ((const orc_obrick*)a)->key, y = ((const orc_obrick*)b)->key;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* sorted unique brick set (Morton order) */
typedef struct {
    orc_obrick* v;
    int64_t n, cap;
} orc_bset;

static void orc_bset_add(orc_bset* s, int64_t x, int64_t y, int64_t z)
{
    if (s->n == s->cap) {
        s->cap = s->cap ? 2 * s->cap : 1024;
        s->v = (orc_obrick*)realloc(s->v, sizeof(orc_obrick) * (size_t)s->cap);
    }
    s->v[s->n].key = orc_morton(x, y, z);
    s->v[s->n].c[0] = x;
    s->v[s->n].c[1] = y;
    s->v[s->n].c[2] = z;
    s->n++;
}

static void orc_bset_finish(orc_bset* s)
{
    qsort(s->v, (size_t)s->n, sizeof(orc_obrick), orc_obrick_cmp);
    int64_t u = 0;
    for (int64_t k = 0; k < s->n; ++k)
        if (k == 0 || s->v[k].key != s->v[u - 1].key) s->v[u++] = s->v[k];
    s->n = u;
}

static int orc_bset_has(const orc_bset* s, uint64_t key)
{
    int64_t lo = 0, hi = s->n - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (s->v[mid].key == key) return 1;
        if (s->v[mid].key < key) lo = mid + 1;
        else hi = mid - 1;
    }
    return 0;
}

/* 26-dilation of s inside [0, nbr)^3 (bricks per axis at that level) */
static orc_bset orc_bset_dilate(const orc_bset* s, int64_t nbr)
{
    orc_bset o = {0, 0, 0};
    for (int64_t k = 0; k < s->n; ++k)
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int64_t x = s->v[k].c[0] + dx, y = s->v[k].c[1] + dy, z = s->v[k].c[2] + dz;
                    if (x < 0 || y < 0 || z < 0 || x >= nbr || y >= nbr || z >= nbr) continue;
                    orc_bset_add(&o, x, y, z);
                }
    orc_bset_finish(&o);
    return o;
}

/*
 * Whole build for nmaps maps of W x H (depth: nmaps * W * H floats, cams: 17
 * doubles each).  Level l = d - dmin, nlev = dmax - dmin + 1.
 * counts[2 * l] = active bricks, counts[2 * l + 1] = frozen bricks of level l.
 * With out != NULL, writes for each level its active then frozen brick
 * coordinates (3 int32 each), levels one after another.  Returns the number of
 * samples.
 */
int64_t orc_octree_build(int nmaps, const double* cams, int W, int H, const float* depth, const double* root_min,
                         double root_edge, int dmin, int dmax, int band, int64_t* counts, int32_t* out)
{
    int nlev = dmax - dmin + 1;
    orc_bset* act = (orc_bset*)calloc((size_t)nlev, sizeof(orc_bset));
    int32_t* dd = (int32_t*)malloc(sizeof(int32_t) * (size_t)W * (size_t)H);
    int64_t* qq = (int64_t*)malloc(sizeof(int64_t) * 3 * (size_t)W * (size_t)H);
    int64_t ns = 0;
    for (int k = 0; k < nmaps; ++k) {
        ns += orc_octree_samples(cams + 17 * k, W, H, depth + (int64_t)k * W * H, root_min, root_edge, dmin, dmax, dd, qq,
                                 NULL);
        for (int64_t p = 0; p < (int64_t)W * H; ++p)
            if (dd[p] >= 0) orc_bset_add(&act[dd[p] - dmin], qq[3 * p] >> 3, qq[3 * p + 1] >> 3, qq[3 * p + 2] >> 3);
    }
    free(dd);
    free(qq);
    for (int l = 0; l < nlev; ++l) {
        orc_bset_finish(&act[l]);
        int64_t nbr = ((int64_t)1 << (dmin + l)) >> 3;
        if (nbr < 1) nbr = 1;
        for (int b = 0; b < band; ++b) {
            orc_bset o = orc_bset_dilate(&act[l], nbr);
            free(act[l].v);
            act[l] = o;
        }
    }
    for (int l = nlev - 1; l >= 1; --l) {
        orc_bset par = {0, 0, 0};
        for (int64_t k = 0; k < act[l].n; ++k)
            orc_bset_add(&par, act[l].v[k].c[0] >> 1, act[l].v[k].c[1] >> 1, act[l].v[k].c[2] >> 1);
        orc_bset_finish(&par);
        int64_t nbr = ((int64_t)1 << (dmin + l - 1)) >> 3;
        if (nbr < 1) nbr = 1;
        orc_bset dl = orc_bset_dilate(&par, nbr);
        for (int64_t k = 0; k < dl.n; ++k) orc_bset_add(&act[l - 1], dl.v[k].c[0], dl.v[k].c[1], dl.v[k].c[2]);
        orc_bset_finish(&act[l - 1]);
        free(par.v);
        free(dl.v);
    }
    int64_t o = 0;
    for (int l = 0; l < nlev; ++l) {
        int64_t nbr = ((int64_t)1 << (dmin + l)) >> 3;
        if (nbr < 1) nbr = 1;
        orc_bset frz = {0, 0, 0};
        if (l > 0) {
            orc_bset dl = orc_bset_dilate(&act[l], nbr);
            for (int64_t k = 0; k < dl.n; ++k)
                if (!orc_bset_has(&act[l], dl.v[k].key)) orc_bset_add(&frz, dl.v[k].c[0], dl.v[k].c[1], dl.v[k].c[2]);
            free(dl.v);
            orc_bset_finish(&frz);
        }
        counts[2 * l] = act[l].n;
        counts[2 * l + 1] = frz.n;
        if (out) {
            for (int64_t k = 0; k < act[l].n; ++k)
                for (int a = 0; a < 3; ++a) out[o++] = (int32_t)act[l].v[k].c[a];
            for (int64_t k = 0; k < frz.n; ++k)
                for (int a = 0; a < 3; ++a) out[o++] = (int32_t)frz.v[k].c[a];
        }
        free(frz.v);
    }
    for (int l = 0; l < nlev; ++l) free(act[l].v);
    free(act);
    return ns;
}
