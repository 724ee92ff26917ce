// Depth pyramids and per-voxel visibility histograms (Sec. 3.4, Alg. 1).
//
// Pyramid: level 0 is the input with invalid samples (NaN, inf, <= 0) made
// NaN; level l+1 has ceil(W_l/2) x ceil(H_l/2) pixels, each the minimum of
// its existing valid children (NaN if none).  Levels go up to
// Lmax = floor(log2(max(W, H))).  One launch per level covers every map of a
// batch.
//
// Cameras: pinhole maps (z-depth) and spherical maps (LIDAR scans, range), see
// tgv_camera.
//
// Histograms: one CTA per active brick, one thread per voxel; each thread
// evaluates Alg. 1 for every map of the batch (gather form: the voxel's own
// projection selects the map's level of detail and pixel), counts its votes
// in registers as packed 16-bit pairs and adds them to its own histogram
// words once.  No atomics: a voxel's words belong to one thread.
//
// The bin decision is taken in FP32 with one rounding per operation, in the
// order listed in Alg1Cam's comment (the __f*_rn intrinsics are never
// contracted into FMAs).
#include <math.h>

#include <algorithm>
#include <vector>

#include "tgv_internal.cuh"

#define TGV_MAX_LEVELS 16

namespace {

// FP32 camera of one map (parameters rounded once from FP64).
// Decision for a voxel with global index idx (per axis):
//   X = o + ((float)idx + 0.5) * h;  d = X - C
//   Xc = (R0 d0 + R1 d1) + R2 d2 (likewise Yc, Zc)
//   pinhole:   requires Zc > 0;  x = (fx Xc)/Zc + cx;  y = (fy Yc)/Zc + cy;
//              diameter fp = (fx (2r))/Zc;  distance dist = Zc
//   spherical: s2 = Xc Xc + Yc Yc;  rho = sqrt(s2 + Zc Zc), requires rho > 0;
//              phi = atan2p(Yc, Xc);  theta = atan2p(Zc, sqrt(s2));
//              x = fx phi + cx;  y = cy - fy theta;  fp = (fx (2r))/rho;  dist = rho
//   LOD l = largest l <= Lmax with 2^l <= max(1, fp)
//   pixel (floor(x 2^-l), floor(y 2^-l)) inside level l, depth valid
//   a = depth - dist;  a >= -eta;  bin = min(floor(((clamp(a/delta) + 1)/2) n), n-1)
struct Alg1Cam {
    float fx, fy, cx, cy, R[9], C[3];
    uint32_t vote;
    int model;  // TGV_PINHOLE / TGV_SPHERICAL
};

// atan2 for the spherical projection: the arctangent polynomial of Abramowitz &
// Stegun 4.4.49 (Hastings; |error| <= 2e-8 on [0, 1]) on t = min/max of |y|, |x|,
// Horner from the highest power, then the octant is restored:
//   |y| > |x|: pi/2 - r;  x < 0: pi - r;  y < 0: -r.   atan2p(0, 0) = 0.
__device__ __forceinline__ float atan2p(float y, float x)
{
    const float ax = fabsf(x), ay = fabsf(y);
    const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
    if (mx == 0.0f) return 0.0f;
    const float t = __fdiv_rn(mn, mx);
    const float s = __fmul_rn(t, t);
    float p = 0.0028662257f;
    p = __fadd_rn(__fmul_rn(p, s), -0.0161657367f);
    p = __fadd_rn(__fmul_rn(p, s), 0.0429096138f);
    p = __fadd_rn(__fmul_rn(p, s), -0.0752896400f);
    p = __fadd_rn(__fmul_rn(p, s), 0.1065626393f);
    p = __fadd_rn(__fmul_rn(p, s), -0.1420889944f);
    p = __fadd_rn(__fmul_rn(p, s), 0.1999355085f);
    p = __fadd_rn(__fmul_rn(p, s), -0.3333314528f);
    p = __fadd_rn(__fmul_rn(p, s), 1.0f);
    float r = __fmul_rn(t, p);
    if (ay > ax) r = __fsub_rn(1.5707963267948966f, r);
    if (x < 0.0f) r = __fsub_rn(3.14159265358979323846f, r);
    return y < 0.0f ? -r : r;
}

struct PyrLayout {
    int nlev;
    int w[TGV_MAX_LEVELS], h[TGV_MAX_LEVELS];
    int64_t off[TGV_MAX_LEVELS];
    int64_t size;  // floats per map
};

struct AccArgs {
    uint32_t* hist;
    const int32_t* coords;  // 3*nb brick coordinates
    const float* pyr;       // nmaps * size floats
    int64_t nb;
    int nmaps, nbins, npairs;
    float o[3], h, r;
    PyrLayout L;
    Alg1Cam cam[TGV_MAPS_PER_LAUNCH];
};

__global__ void pyr_level0_kernel(const float* __restrict__ depth, int64_t pitch, int64_t stride, int W, int H,
                                  float* __restrict__ pyr, int64_t size, int nmaps)
{
    const int64_t n = (int64_t)W * H;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n * nmaps;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = g / n, k = g - m * n;
        const int64_t j = k / W, i = k - j * W;
        float dv = depth[m * stride + j * pitch + i];
        pyr[m * size + k] = (isfinite(dv) && dv > 0.0f) ? dv : __int_as_float(0x7fc00000);
    }
}

__global__ void pyr_down_kernel(float* __restrict__ pyr, int64_t size, int nmaps, int64_t src_off, int ws, int hs,
                                int64_t dst_off, int wd, int hd)
{
    const int64_t n = (int64_t)wd * hd;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n * nmaps;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = g / n, k = g - m * n;
        const int j = (int)(k / wd), i = (int)(k - (int64_t)j * wd);
        const float* src = pyr + m * size + src_off;
        float best = __int_as_float(0x7fc00000);
#pragma unroll
        for (int dj = 0; dj < 2; ++dj)
#pragma unroll
            for (int di = 0; di < 2; ++di) {
                const int ci = 2 * i + di, cj = 2 * j + dj;
                if (ci < ws && cj < hs) {
                    const float c = src[(int64_t)cj * ws + ci];
                    if (!isnan(c) && (isnan(best) || c < best)) best = c;
                }
            }
        pyr[m * size + dst_off + k] = best;
    }
}

// Alg. 1 up to the depth read: LOD level l and pixel (i, j) of the voxel centre X,
// and its distance to the camera.  false: not projected into the map.
__device__ __forceinline__ bool alg1_pixel(const Alg1Cam& c, const PyrLayout& L, const float X[3], float diam,
                                           int& l, int& i, int& j, float& dist)
{
    const float d0 = __fsub_rn(X[0], c.C[0]);
    const float d1 = __fsub_rn(X[1], c.C[1]);
    const float d2 = __fsub_rn(X[2], c.C[2]);
    const float zc = __fadd_rn(__fadd_rn(__fmul_rn(c.R[6], d0), __fmul_rn(c.R[7], d1)), __fmul_rn(c.R[8], d2));
    if (c.model == TGV_PINHOLE && !(zc > 0.0f)) return false;
    const float xc = __fadd_rn(__fadd_rn(__fmul_rn(c.R[0], d0), __fmul_rn(c.R[1], d1)), __fmul_rn(c.R[2], d2));
    const float yc = __fadd_rn(__fadd_rn(__fmul_rn(c.R[3], d0), __fmul_rn(c.R[4], d1)), __fmul_rn(c.R[5], d2));
    float px, py, fp;
    if (c.model == TGV_PINHOLE) {
        px = __fadd_rn(__fdiv_rn(__fmul_rn(c.fx, xc), zc), c.cx);
        py = __fadd_rn(__fdiv_rn(__fmul_rn(c.fy, yc), zc), c.cy);
        fp = __fdiv_rn(__fmul_rn(c.fx, diam), zc);
        dist = zc;
    } else {
        const float s2 = __fadd_rn(__fmul_rn(xc, xc), __fmul_rn(yc, yc));
        const float rho = __fsqrt_rn(__fadd_rn(s2, __fmul_rn(zc, zc)));
        if (!(rho > 0.0f)) return false;
        const float phi = atan2p(yc, xc);
        const float theta = atan2p(zc, __fsqrt_rn(s2));
        px = __fadd_rn(__fmul_rn(c.fx, phi), c.cx);
        py = __fsub_rn(c.cy, __fmul_rn(c.fy, theta));
        fp = __fdiv_rn(__fmul_rn(c.fx, diam), rho);
        dist = rho;
    }
    l = 0;
    float p2 = 2.0f;
    while (l + 1 < L.nlev && p2 <= fp) {
        ++l;
        p2 = __fmul_rn(p2, 2.0f);
    }
    const float scale = __int_as_float((127 - l) << 23);  // exactly 2^-l
    const float xl = __fmul_rn(px, scale), yl = __fmul_rn(py, scale);
    if (!(xl >= 0.0f && xl < (float)L.w[l])) return false;
    if (!(yl >= 0.0f && yl < (float)L.h[l])) return false;
    i = (int)xl;  // truncation == floor for non-negative values
    j = (int)yl;
    return true;
}

// Alg. 1 after the depth read: the bin of a = depth - dist, or -1 (no sample, or
// occluded beyond eta)
__device__ __forceinline__ int alg1_bin_of(float depth, float dist, float delta, float eta, int nbins)
{
    if (isnan(depth)) return -1;
    const float a = __fsub_rn(depth, dist);
    if (a < -eta) return -1;
    float ac = __fdiv_rn(a, delta);
    ac = fminf(1.0f, ac);
    ac = fmaxf(-1.0f, ac);
    const float t1 = __fadd_rn(ac, 1.0f);
    const float t2 = __fmul_rn(t1, 0.5f);  // = t1 / 2 exactly (a power of two)
    const float t3 = __fmul_rn(t2, (float)nbins);
    int bin = (int)floorf(t3);
    return bin > nbins - 1 ? nbins - 1 : bin;
}

__device__ __forceinline__ int alg1_bin(const Alg1Cam& c, const PyrLayout& L, const float* __restrict__ pyr,
                                        const float X[3], float diam, float delta, float eta, int nbins)
{
    int l, i, j;
    float dist;
    if (!alg1_pixel(c, L, X, diam, l, i, j, dist)) return -1;
    const float depth = __ldg(pyr + L.off[l] + (int64_t)j * L.w[l] + i);
    return alg1_bin_of(depth, dist, delta, eta, nbins);
}

__global__ void __launch_bounds__(512) hist_accumulate_kernel(const AccArgs A)
{
    __shared__ int32_t s_c[3];
    const int64_t b = blockIdx.x;
    const int t = threadIdx.x;
    if (t < 3) s_c[t] = A.coords[3 * b + t];
    __syncthreads();
    const int loc[3] = {t & 7, (t >> 3) & 7, t >> 6};
    float X[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int idx = 8 * s_c[a] + loc[a];
        X[a] = __fadd_rn(A.o[a], __fmul_rn(__fadd_rn(__int2float_rn(idx), 0.5f), A.h));
    }
    const float diam = __fmul_rn(A.r, 2.0f);
    const float delta = __fmul_rn(6.0f, A.r);
    const float eta = __fmul_rn(3.0f, delta);
    // this thread's packed counts of the launch, in shared memory so that a vote is
    // one indexed add (column t of word k: no two threads share a word)
    __shared__ uint32_t s_acc[TGV_MAX_BINS / 2][TGV_BVOX];
#pragma unroll
    for (int k = 0; k < TGV_MAX_BINS / 2; ++k) s_acc[k][t] = 0u;
    for (int m = 0; m < A.nmaps; ++m) {
        const int bin = alg1_bin(A.cam[m], A.L, A.pyr + (int64_t)m * A.L.size, X, diam, delta, eta, A.nbins);
        if (bin >= 0) s_acc[bin >> 1][t] += A.cam[m].vote << ((bin & 1) * 16);
    }
    for (int k = 0; k < A.npairs; ++k) {
        const uint32_t a = s_acc[k][t];
        if (a != 0u) {
            uint32_t* w = A.hist + ((int64_t)b * A.npairs + k) * TGV_BVOX + t;
            *w += a;
        }
    }
}

// ---- scatter form: one thread per pyramid pixel (map m, level l, pixel (i, j))
//
// The voxels whose Alg. 1 decision lands on (l, i, j) have their centres inside
// the pixel's frustum (the cone from the camera centre through the level-0 square
// [i 2^l, (i+1) 2^l) x [j 2^l, (j+1) 2^l)), at camera depths zc where the LOD is l
// (2^l <= fx 2r / zc < 2^(l+1), open at the first and last level) and not beyond
// the pixel's depth + eta.  The thread walks the voxel-centre planes across the
// dominant axis of the pixel's central ray inside that depth window; in each
// plane the frustum's cross-section is the quadrilateral of its four corner rays,
// whose bounding box (plus a margin far above FP32 rounding) holds every
// candidate.  A pixel whose corner rays run too close to the planes (the widest
// pixels of the coarsest levels, whose depth window lies next to the camera)
// takes the bounding box of the whole window instead.  Each candidate repeats the
// decision of the gather form (same FP32 operations); the voxel is counted only
// if the decision picks this level and pixel, so every (voxel, map) pair is
// counted once, as in the gather form, and the integer counts are identical.
struct ScatArgs {
    uint32_t* hist;
    const int32_t* grid;  // active brick index per brick cell of the bounding box, -1 none
    int gmin[3], gdim[3];
    const float* pyr;
    int nmaps, nbins, npairs;
    float o[3], h, r;
    PyrLayout L;
    float zdom[TGV_MAPS_PER_LAUNCH][2];  // camera depth range of the voxel centres' box
    Alg1Cam cam[TGV_MAPS_PER_LAUNCH];
};

// world direction of the ray through level-0 pixel coordinates (px, py), zc = 1
__device__ __forceinline__ void pix_dir(const Alg1Cam& c, float px, float py, float d[3])
{
    const float xn = (px - c.cx) / c.fx, yn = (py - c.cy) / c.fy;
#pragma unroll
    for (int a = 0; a < 3; ++a) d[a] = c.R[a] * xn + c.R[3 + a] * yn + c.R[6 + a];
}

__global__ void __launch_bounds__(256) hist_scatter_kernel(const ScatArgs A)
{
    const int64_t per_map = A.L.size;
    const float diam = __fmul_rn(A.r, 2.0f);
    const float delta = __fmul_rn(6.0f, A.r);
    const float eta = __fmul_rn(3.0f, delta);
    const float mg = 0.05f * A.h;  // geometric margin, in world units
    int vlo[3], vhi[3];            // voxel index range of the box
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        vlo[a] = 8 * A.gmin[a];
        vhi[a] = 8 * (A.gmin[a] + A.gdim[a]) - 1;
    }
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < per_map * A.nmaps;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int m = (int)(g / per_map);
        const int64_t k = g - (int64_t)m * per_map;
        const float D = A.pyr[g];
        if (isnan(D)) continue;
        int l = 0;
        while (l + 1 < A.L.nlev && A.L.off[l + 1] <= k) ++l;
        const int64_t kk = k - A.L.off[l];
        const int pj = (int)(kk / A.L.w[l]), pi = (int)(kk - (int64_t)pj * A.L.w[l]);
        const Alg1Cam& c = A.cam[m];
        // depth window
        const float F = c.fx * diam;
        float zlo = l + 1 < A.L.nlev ? F * __int_as_float((127 - l - 1) << 23) : 0.0f;
        float zhi = l > 0 ? F * __int_as_float((127 - l) << 23) : INFINITY;
        zlo = fmaxf(fmaxf(zlo * (1.0f - 1e-4f), A.zdom[m][0]), 0.0f);
        zhi = fminf(fminf(zhi * (1.0f + 1e-4f), (D + eta) * (1.0f + 1e-4f) + mg), A.zdom[m][1]);
        if (!(zlo < zhi)) continue;
        // corner rays of the pixel and its central ray
        const float s = __int_as_float((127 + l) << 23);
        float dq[4][3], dc[3];
#pragma unroll
        for (int q = 0; q < 4; ++q) pix_dir(c, (pi + (q & 1)) * s, (pj + (q >> 1)) * s, dq[q]);
        pix_dir(c, (pi + 0.5f) * s, (pj + 0.5f) * s, dc);
        int ax = 0;
        if (fabsf(dc[1]) > fabsf(dc[ax])) ax = 1;
        if (fabsf(dc[2]) > fabsf(dc[ax])) ax = 2;
        bool well = true;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float n = sqrtf(dq[q][0] * dq[q][0] + dq[q][1] * dq[q][1] + dq[q][2] * dq[q][2]);
            well = well && (dq[q][ax] > 0.0f) == (dc[ax] > 0.0f) && fabsf(dq[q][ax]) >= 0.25f * n;
        }
        auto visit = [&](int gx, int gy, int gz) {
            const int gidx[3] = {gx, gy, gz};
            int cell = 0;
#pragma unroll
            for (int a = 2; a >= 0; --a) {
                const int bc = (gidx[a] >> 3) - A.gmin[a];
                if (bc < 0 || bc >= A.gdim[a]) return;
                cell = cell * A.gdim[a] + bc;
            }
            const int32_t b = A.grid[cell];
            if (b < 0) return;
            float X[3];
#pragma unroll
            for (int a = 0; a < 3; ++a)
                X[a] = __fadd_rn(A.o[a], __fmul_rn(__fadd_rn(__int2float_rn(gidx[a]), 0.5f), A.h));
            int l2, i2, j2;
            float dist;
            if (!alg1_pixel(c, A.L, X, diam, l2, i2, j2, dist)) return;
            if (l2 != l || i2 != pi || j2 != pj) return;
            const int bin = alg1_bin_of(D, dist, delta, eta, A.nbins);
            if (bin < 0) return;
            const int loc = (gx & 7) + 8 * (gy & 7) + 64 * (gz & 7);
            atomicAdd(A.hist + ((int64_t)b * A.npairs + (bin >> 1)) * TGV_BVOX + loc, c.vote << ((bin & 1) * 16));
        };
        auto lo_idx = [&](float x, int a) { return (int)ceilf((x - mg - A.o[a]) / A.h - 0.5f); };
        auto hi_idx = [&](float x, int a) { return (int)floorf((x + mg - A.o[a]) / A.h - 0.5f); };
        if (well) {
            // planes of voxel centres across axis ax within the window; b1, b2 are the
            // other two axes (components picked into registers, no indexed arrays)
            const int b1 = ax == 0 ? 1 : 0, b2 = ax == 2 ? 1 : 2;
            auto pick = [](const float* v, int a) { return a == 0 ? v[0] : (a == 1 ? v[1] : v[2]); };
            float da[4], d1[4], d2[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                da[q] = pick(dq[q], ax);
                d1[q] = pick(dq[q], b1);
                d2[q] = pick(dq[q], b2);
            }
            const float Ca = pick(c.C, ax), C1 = pick(c.C, b1), C2 = pick(c.C, b2);
            const float oa = pick(A.o, ax);
            float lo = INFINITY, hi = -INFINITY;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float x0 = Ca + zlo * da[q], x1 = Ca + zhi * da[q];
                lo = fminf(lo, fminf(x0, x1));
                hi = fmaxf(hi, fmaxf(x0, x1));
            }
            const int vla = ax == 0 ? vlo[0] : (ax == 1 ? vlo[1] : vlo[2]);
            const int vha = ax == 0 ? vhi[0] : (ax == 1 ? vhi[1] : vhi[2]);
            const int k0 = max((int)ceilf((lo - mg - oa) / A.h - 0.5f), vla);
            const int k1 = min((int)floorf((hi + mg - oa) / A.h - 0.5f), vha);
            const float o1 = pick(A.o, b1), o2 = pick(A.o, b2);
            const int vl1 = b1 == 0 ? vlo[0] : vlo[1], vh1 = b1 == 0 ? vhi[0] : vhi[1];
            const int vl2 = b2 == 2 ? vlo[2] : vlo[1], vh2 = b2 == 2 ? vhi[2] : vhi[1];
            for (int kp = k0; kp <= k1; ++kp) {
                const float P = oa + (kp + 0.5f) * A.h;
                float l1 = INFINITY, h1 = -INFINITY, l2 = INFINITY, h2 = -INFINITY;
                bool front = true;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float z = (P - Ca) / da[q];
                    front = front && z > 0.0f;
                    const float y1 = C1 + z * d1[q], y2 = C2 + z * d2[q];
                    l1 = fminf(l1, y1);
                    h1 = fmaxf(h1, y1);
                    l2 = fminf(l2, y2);
                    h2 = fmaxf(h2, y2);
                }
                if (!front) continue;
                const int i1 = max((int)ceilf((l1 - mg - o1) / A.h - 0.5f), vl1);
                const int j1 = min((int)floorf((h1 + mg - o1) / A.h - 0.5f), vh1);
                const int i2 = max((int)ceilf((l2 - mg - o2) / A.h - 0.5f), vl2);
                const int j2 = min((int)floorf((h2 + mg - o2) / A.h - 0.5f), vh2);
                for (int u2 = i2; u2 <= j2; ++u2)
                    for (int u1 = i1; u1 <= j1; ++u1) {
                        const int gx = ax == 0 ? kp : u1;
                        const int gy = ax == 1 ? kp : (ax == 0 ? u1 : u2);
                        const int gz = ax == 2 ? kp : u2;
                        visit(gx, gy, gz);
                    }
            }
        } else {
            // bounding box of the frustum between the window's two depths
            float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float x0 = c.C[a] + zlo * dq[q][a], x1 = c.C[a] + zhi * dq[q][a];
                    lo[a] = fminf(lo[a], fminf(x0, x1));
                    hi[a] = fmaxf(hi[a], fmaxf(x0, x1));
                }
            int r0[3], r1[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                r0[a] = max(lo_idx(lo[a], a), vlo[a]);
                r1[a] = min(hi_idx(hi[a], a), vhi[a]);
            }
            for (int gz = r0[2]; gz <= r1[2]; ++gz)
                for (int gy = r0[1]; gy <= r1[1]; ++gy)
                    for (int gx = r0[0]; gx <= r1[0]; ++gx) visit(gx, gy, gz);
        }
    }
}

PyrLayout make_layout(int W, int H)
{
    PyrLayout L;
    int m = W > H ? W : H, lmax = 0;
    while ((1 << (lmax + 1)) <= m) ++lmax;
    L.nlev = lmax + 1;
    int64_t off = 0;
    int w = W, h = H;
    for (int l = 0; l < L.nlev; ++l) {
        L.w[l] = w;
        L.h[l] = h;
        L.off[l] = off;
        off += (int64_t)w * h;
        w = (w + 1) / 2;
        h = (h + 1) / 2;
    }
    L.size = off;
    return L;
}

unsigned grid_for(tgv_domain* d, int64_t n, int block)
{
    int64_t g = (n + block - 1) / block;
    int64_t cap = (int64_t)d->sm_count * 16;
    if (g > cap) g = cap;
    return (unsigned)(g < 1 ? 1 : g);
}

// Brick index of every brick cell of the active bricks' bounding box (scatter form),
// built on first use; a level's bricks do not change after creation.
tgv_status build_brick_grid(tgv_domain* d, TgvLevel& L)
{
    if (L.bgrid || L.nb == 0) return TGV_OK;
    int64_t mn[3], mx[3];
    for (int a = 0; a < 3; ++a) mn[a] = mx[a] = L.coords[a];
    for (int64_t b = 1; b < L.nb; ++b)
        for (int a = 0; a < 3; ++a) {
            mn[a] = std::min<int64_t>(mn[a], L.coords[3 * b + a]);
            mx[a] = std::max<int64_t>(mx[a], L.coords[3 * b + a]);
        }
    int64_t cells = 1;
    for (int a = 0; a < 3; ++a) cells *= mx[a] - mn[a] + 1;
    if (cells > ((int64_t)1 << 28) || mn[0] < -(1 << 27) || mx[0] >= (1 << 27) || mn[1] < -(1 << 27) ||
        mx[1] >= (1 << 27) || mn[2] < -(1 << 27) || mx[2] >= (1 << 27))
        return tgv_fail(d, TGV_ERR_UNSUPPORTED, "scatter-form histograms: the bricks' bounding box is too large");
    std::vector<int32_t> grid((size_t)cells, -1);
    for (int64_t b = 0; b < L.nb; ++b) {
        const int64_t x = L.coords[3 * b] - mn[0], y = L.coords[3 * b + 1] - mn[1], z = L.coords[3 * b + 2] - mn[2];
        grid[(size_t)((z * (mx[1] - mn[1] + 1) + y) * (mx[0] - mn[0] + 1) + x)] = (int32_t)b;
    }
    for (int a = 0; a < 3; ++a) {
        L.bgmin[a] = (int32_t)mn[a];
        L.bgdim[a] = (int32_t)(mx[a] - mn[a] + 1);
    }
    cudaError_t e = cudaMalloc(&L.bgrid, grid.size() * 4);
    if (e != cudaSuccess) {
        cudaGetLastError();
        L.bgrid = nullptr;
        return tgv_fail(d, TGV_ERR_OUT_OF_MEMORY, "brick grid allocation failed");
    }
    d->bytes += (int64_t)grid.size() * 4;
    e = cudaMemcpyAsync(L.bgrid, grid.data(), grid.size() * 4, cudaMemcpyHostToDevice, d->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    return tgv_cuda_check(d, e, "brick grid upload");
}

}  // namespace

tgv_status tgv_launch_accumulate(tgv_domain* d, TgvLevel& Lv, const tgv_camera* cams, int nmaps, const float* depth,
                                 int64_t pitch, int64_t stride, const uint32_t* votes)
{
    const int W = cams[0].width, H = cams[0].height;
    const PyrLayout L = make_layout(W, H);
    const bool scatter = d->prm.hist_form == TGV_HIST_SCATTER;
    if (scatter) {
        for (int m = 0; m < nmaps; ++m)
            if (cams[m].model != TGV_PINHOLE)
                return tgv_fail(d, TGV_ERR_UNSUPPORTED, "scatter-form histograms take pinhole maps only");
        if (Lv.nb == 0) return TGV_OK;
        tgv_status st = build_brick_grid(d, Lv);
        if (st != TGV_OK) return st;
    }
    for (int m0 = 0; m0 < nmaps; m0 += TGV_MAPS_PER_LAUNCH) {
        const int nm = nmaps - m0 < TGV_MAPS_PER_LAUNCH ? nmaps - m0 : TGV_MAPS_PER_LAUNCH;
        tgv_status st = tgv_scratch(d, d->pyr, sizeof(float) * (size_t)L.size * nm);
        if (st != TGV_OK) return st;
        float* pyr = (float*)d->pyr.ptr;
        const int64_t n0 = (int64_t)W * H * nm;
        pyr_level0_kernel<<<grid_for(d, n0, 256), 256, 0, d->stream>>>(depth + (int64_t)m0 * stride, pitch, stride, W,
                                                                       H, pyr, L.size, nm);
        d->launches++;
        for (int l = 1; l < L.nlev; ++l) {
            const int64_t n = (int64_t)L.w[l] * L.h[l] * nm;
            pyr_down_kernel<<<grid_for(d, n, 256), 256, 0, d->stream>>>(pyr, L.size, nm, L.off[l - 1], L.w[l - 1],
                                                                        L.h[l - 1], L.off[l], L.w[l], L.h[l]);
            d->launches++;
        }
        AccArgs A;
        A.hist = Lv.hist;
        A.coords = nullptr;
        A.pyr = pyr;
        A.nb = Lv.nb;
        A.nmaps = nm;
        A.nbins = d->prm.nbins;
        A.npairs = (d->prm.nbins + 1) / 2;
        for (int a = 0; a < 3; ++a) A.o[a] = (float)Lv.origin[a];
        A.h = (float)Lv.h;
        A.r = (float)Lv.radius;
        A.L = L;
        for (int m = 0; m < nm; ++m) {
            const tgv_camera& c = cams[m0 + m];
            Alg1Cam& g = A.cam[m];
            g.fx = (float)c.fx;
            g.fy = (float)c.fy;
            g.cx = (float)c.cx;
            g.cy = (float)c.cy;
            for (int k = 0; k < 9; ++k) g.R[k] = (float)c.R[k];
            for (int k = 0; k < 3; ++k) g.C[k] = (float)c.C[k];
            g.vote = votes ? votes[m0 + m] : 1u;
            g.model = c.model;
        }
        A.coords = Lv.coords_dev;
        if (!scatter) {
            hist_accumulate_kernel<<<(unsigned)Lv.nb, TGV_BVOX, 0, d->stream>>>(A);
        } else {
            ScatArgs S;
            S.hist = Lv.hist;
            S.grid = Lv.bgrid;
            for (int a = 0; a < 3; ++a) {
                S.gmin[a] = Lv.bgmin[a];
                S.gdim[a] = Lv.bgdim[a];
                S.o[a] = A.o[a];
            }
            S.pyr = pyr;
            S.nmaps = nm;
            S.nbins = A.nbins;
            S.npairs = A.npairs;
            S.h = A.h;
            S.r = A.r;
            S.L = L;
            for (int m = 0; m < nm; ++m) {
                S.cam[m] = A.cam[m];
                // camera depth range of the box of voxel centres (its 8 corners), widened
                const tgv_camera& c = cams[m0 + m];
                double zmin = INFINITY, zmax = -INFINITY;
                for (int corner = 0; corner < 8; ++corner) {
                    double zc = 0.0;
                    for (int a = 0; a < 3; ++a) {
                        const int64_t vi = (corner >> a) & 1 ? 8 * ((int64_t)Lv.bgmin[a] + Lv.bgdim[a]) - 1
                                                             : 8 * (int64_t)Lv.bgmin[a];
                        const double X = Lv.origin[a] + ((double)vi + 0.5) * Lv.h;
                        zc += c.R[6 + a] * (X - c.C[a]);
                    }
                    zmin = std::min(zmin, zc);
                    zmax = std::max(zmax, zc);
                }
                const double pad = 0.05 * Lv.h + 1e-5 * (fabs(zmin) + fabs(zmax));
                S.zdom[m][0] = (float)(zmin - pad);
                S.zdom[m][1] = (float)(zmax + pad);
            }
            hist_scatter_kernel<<<grid_for(d, (int64_t)nm * L.size, 256), 256, 0, d->stream>>>(S);
        }
        d->launches++;
        st = tgv_cuda_check(d, cudaGetLastError(), scatter ? "hist_scatter_kernel launch" : "hist_accumulate_kernel launch");
        if (st != TGV_OK) return st;
    }
    return TGV_OK;
}
