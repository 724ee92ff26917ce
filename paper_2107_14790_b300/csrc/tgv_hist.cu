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

__device__ __forceinline__ int alg1_bin(const Alg1Cam& c, const PyrLayout& L, const float* __restrict__ pyr,
                                        const float X[3], float diam, float delta, float eta, int nbins)
{
    const float d0 = __fsub_rn(X[0], c.C[0]);
    const float d1 = __fsub_rn(X[1], c.C[1]);
    const float d2 = __fsub_rn(X[2], c.C[2]);
    const float zc = __fadd_rn(__fadd_rn(__fmul_rn(c.R[6], d0), __fmul_rn(c.R[7], d1)), __fmul_rn(c.R[8], d2));
    if (c.model == TGV_PINHOLE && !(zc > 0.0f)) return -1;
    const float xc = __fadd_rn(__fadd_rn(__fmul_rn(c.R[0], d0), __fmul_rn(c.R[1], d1)), __fmul_rn(c.R[2], d2));
    const float yc = __fadd_rn(__fadd_rn(__fmul_rn(c.R[3], d0), __fmul_rn(c.R[4], d1)), __fmul_rn(c.R[5], d2));
    float px, py, fp, dist;
    if (c.model == TGV_PINHOLE) {
        px = __fadd_rn(__fdiv_rn(__fmul_rn(c.fx, xc), zc), c.cx);
        py = __fadd_rn(__fdiv_rn(__fmul_rn(c.fy, yc), zc), c.cy);
        fp = __fdiv_rn(__fmul_rn(c.fx, diam), zc);
        dist = zc;
    } else {
        const float s2 = __fadd_rn(__fmul_rn(xc, xc), __fmul_rn(yc, yc));
        const float rho = __fsqrt_rn(__fadd_rn(s2, __fmul_rn(zc, zc)));
        if (!(rho > 0.0f)) return -1;
        const float phi = atan2p(yc, xc);
        const float theta = atan2p(zc, __fsqrt_rn(s2));
        px = __fadd_rn(__fmul_rn(c.fx, phi), c.cx);
        py = __fsub_rn(c.cy, __fmul_rn(c.fy, theta));
        fp = __fdiv_rn(__fmul_rn(c.fx, diam), rho);
        dist = rho;
    }
    int l = 0;
    float p2 = 2.0f;
    while (l + 1 < L.nlev && p2 <= fp) {
        ++l;
        p2 = __fmul_rn(p2, 2.0f);
    }
    const float scale = __int_as_float((127 - l) << 23);  // exactly 2^-l
    const float xl = __fmul_rn(px, scale), yl = __fmul_rn(py, scale);
    const int wl = L.w[l], hl = L.h[l];
    if (!(xl >= 0.0f && xl < (float)wl)) return -1;
    if (!(yl >= 0.0f && yl < (float)hl)) return -1;
    const int i = (int)xl, j = (int)yl;  // truncation == floor for non-negative values
    const float depth = __ldg(pyr + L.off[l] + (int64_t)j * wl + i);
    if (isnan(depth)) return -1;
    const float a = __fsub_rn(depth, dist);
    if (a < -eta) return -1;
    float ac = __fdiv_rn(a, delta);
    ac = fminf(1.0f, ac);
    ac = fmaxf(-1.0f, ac);
    const float t1 = __fadd_rn(ac, 1.0f);
    const float t2 = __fdiv_rn(t1, 2.0f);
    const float t3 = __fmul_rn(t2, (float)nbins);
    int bin = (int)floorf(t3);
    return bin > nbins - 1 ? nbins - 1 : bin;
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
    uint32_t acc[TGV_MAX_BINS / 2];
#pragma unroll
    for (int k = 0; k < TGV_MAX_BINS / 2; ++k) acc[k] = 0u;
    for (int m = 0; m < A.nmaps; ++m) {
        const int bin = alg1_bin(A.cam[m], A.L, A.pyr + (int64_t)m * A.L.size, X, diam, delta, eta, A.nbins);
        if (bin >= 0) {
            const uint32_t inc = A.cam[m].vote << ((bin & 1) * 16);
#pragma unroll
            for (int k = 0; k < TGV_MAX_BINS / 2; ++k)
                if (k == (bin >> 1)) acc[k] += inc;
        }
    }
#pragma unroll
    for (int k = 0; k < TGV_MAX_BINS / 2; ++k) {
        if (k < A.npairs && acc[k] != 0u) {
            uint32_t* w = A.hist + ((int64_t)b * A.npairs + k) * TGV_BVOX + t;
            *w += acc[k];
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

}  // namespace

tgv_status tgv_launch_accumulate(tgv_domain* d, TgvLevel& Lv, const tgv_camera* cams, int nmaps, const float* depth,
                                 int64_t pitch, int64_t stride, const uint32_t* votes)
{
    const int W = cams[0].width, H = cams[0].height;
    const PyrLayout L = make_layout(W, H);
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
        hist_accumulate_kernel<<<(unsigned)Lv.nb, TGV_BVOX, 0, d->stream>>>(A);
        d->launches++;
        st = tgv_cuda_check(d, cudaGetLastError(), "hist_accumulate_kernel launch");
        if (st != TGV_OK) return st;
    }
    return TGV_OK;
}
