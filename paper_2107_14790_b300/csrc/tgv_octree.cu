// Brick domains from depth maps (Sec. 3.3 Eq. 4, Sec. 4.1-4.2), in memory.
//
// Every valid pixel of a pinhole map is a point sample X (its z-depth
// unprojected) with radius r = half the mean distance to the points of its
// valid 4-neighbours (left, right, up, down).  Eq. 4 puts the sample in the cube
// of depth d with 0.75 r <= r_root 2^-d < 1.5 r: the smallest d in
// [depth_min, depth_max] with r_root 2^-d < 1.5 r (depth_max if none), cube
// q = floor(((X - root_min) / E) 2^d).  All of it in FP32 with one rounding
// per operation (the order is spelled out in the kernels), so the decisions are
// reproducible.  Level l = d - depth_min has voxel edge E / 2^d; its bricks are
// the occupied cubes' q >> 3.
//
// GPU: one pass unprojects a batch of maps, a second computes radius, depth and
// brick key (level << 57 | Morton code of the brick) and inserts the key into a
// device hash set (open addressing, bounded linear probing; a full table is
// detected and the build retried with a larger one).  The unique keys (far fewer
// than the samples) go to the host, which sorts them and forms the levels:
// dilation by `band` rings of 26-neighbours, the 2:1 balance (finest first,
// level l-1 gains the parents b >> 1 of level l's bricks dilated once, so every
// finer level is wrapped by a shell of the next coarser one), and the frozen
// shell of each level above the coarsest (26-neighbours of its active bricks
// that are not active).  Bricks of a level are listed in Morton order.
#include <math.h>

#include <algorithm>
#include <vector>

#include "tgv_internal.cuh"

struct tgv_octree {
    struct Level {
        std::vector<int32_t> active, frozen;  // 3 coordinates per brick
        double origin[3], h;
    };
    std::vector<Level> levels;
    int64_t samples = 0;
};

namespace {

constexpr uint64_t kEmpty = ~(uint64_t)0;
constexpr int kMaxProbe = 4096;

__host__ __device__ __forceinline__ uint64_t spread3(uint64_t v)
{
    // bits 0..20 of v to every third bit
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

__host__ __device__ __forceinline__ uint64_t morton3(uint64_t x, uint64_t y, uint64_t z)
{
    return spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
}

__host__ __device__ __forceinline__ uint64_t compact3(uint64_t v)
{
    v &= 0x1249249249249249ull;
    v = (v | (v >> 2)) & 0x10c30c30c30c30c3ull;
    v = (v | (v >> 4)) & 0x100f00f00f00f00full;
    v = (v | (v >> 8)) & 0x1f0000ff0000ffull;
    v = (v | (v >> 16)) & 0x1f00000000ffffull;
    v = (v | (v >> 32)) & 0x1fffffull;
    return v;
}

// splitmix64 finaliser (Steele, Lea, Flood 2014) as the hash of a key
__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

struct OctCam {
    float fx, fy, cx, cy, R[9], C[3];
};

struct OctArgs {
    const float* depth;
    int64_t pitch, stride;
    int W, H, nmaps;
    OctCam cam[TGV_MAPS_PER_LAUNCH];
    float4* X;  // nmaps * H * W points (w = 1 valid)
    float m[3], E, rroot;
    int dmin, dmax;
    uint64_t* table;
    uint64_t cap;  // power of two
    unsigned long long* counters;  // [0] samples, [1] insert failures
};

__global__ void oct_unproject_kernel(const OctArgs A)
{
    const int64_t n = (int64_t)A.W * A.H;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n * A.nmaps;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int m = (int)(g / n);
        const int64_t p = g - m * n;
        const int j = (int)(p / A.W), i = (int)(p - (int64_t)j * A.W);
        const float z = A.depth[m * A.stride + (int64_t)j * A.pitch + i];
        float4 out = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (isfinite(z) && z > 0.0f) {
            const OctCam& c = A.cam[m];
            const float pc0 = __fmul_rn(__fdiv_rn(__fsub_rn(__fadd_rn(__int2float_rn(i), 0.5f), c.cx), c.fx), z);
            const float pc1 = __fmul_rn(__fdiv_rn(__fsub_rn(__fadd_rn(__int2float_rn(j), 0.5f), c.cy), c.fy), z);
            float x[3];
            for (int a = 0; a < 3; ++a) {
                float s = __fadd_rn(__fmul_rn(c.R[a], pc0), __fmul_rn(c.R[3 + a], pc1));
                s = __fadd_rn(s, __fmul_rn(c.R[6 + a], z));
                x[a] = __fadd_rn(c.C[a], s);
            }
            out = make_float4(x[0], x[1], x[2], 1.0f);
        }
        A.X[g] = out;
    }
}

__global__ void oct_key_kernel(const OctArgs A)
{
    const int64_t n = (int64_t)A.W * A.H;
    unsigned long long mine = 0, fails = 0;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n * A.nmaps;
         g += (int64_t)gridDim.x * blockDim.x) {
        const float4 x = A.X[g];
        if (x.w == 0.0f) continue;
        const int m = (int)(g / n);
        const int64_t p = g - m * n;
        const int j = (int)(p / A.W), i = (int)(p - (int64_t)j * A.W);
        const int di[4] = {-1, 1, 0, 0}, dj[4] = {0, 0, -1, 1};
        float sum = 0.0f;
        int cnt = 0;
        for (int k = 0; k < 4; ++k) {
            const int ii = i + di[k], jj = j + dj[k];
            if (ii < 0 || ii >= A.W || jj < 0 || jj >= A.H) continue;
            const float4 y = A.X[(int64_t)m * n + (int64_t)jj * A.W + ii];
            if (y.w == 0.0f) continue;
            const float e0 = __fsub_rn(y.x, x.x), e1 = __fsub_rn(y.y, x.y), e2 = __fsub_rn(y.z, x.z);
            const float l2 = __fadd_rn(__fadd_rn(__fmul_rn(e0, e0), __fmul_rn(e1, e1)), __fmul_rn(e2, e2));
            sum = __fadd_rn(sum, __fsqrt_rn(l2));
            ++cnt;
        }
        if (cnt == 0) continue;
        const float r = __fmul_rn(0.5f, __fdiv_rn(sum, __int2float_rn(cnt)));
        const float lim = __fmul_rn(1.5f, r);
        int d = A.dmin;
        while (d < A.dmax && !(__fmul_rn(A.rroot, __int_as_float((127 - d) << 23)) < lim)) ++d;
        const float two_d = __int_as_float((127 + d) << 23);
        const float xs[3] = {x.x, x.y, x.z};
        uint64_t q[3];
        bool inside = true;
        for (int a = 0; a < 3; ++a) {
            const float t = __fmul_rn(__fdiv_rn(__fsub_rn(xs[a], A.m[a]), A.E), two_d);
            if (!(t >= 0.0f && t < two_d)) inside = false;
            q[a] = inside ? (uint64_t)floorf(t) : 0;
        }
        if (!inside) continue;
        ++mine;
        const uint64_t key = ((uint64_t)(d - A.dmin) << 57) | morton3(q[0] >> 3, q[1] >> 3, q[2] >> 3);
        uint64_t h = mix64(key) & (A.cap - 1);
        bool done = false;
        for (int probe = 0; probe < kMaxProbe && !done; ++probe) {
            const uint64_t cur = A.table[h];
            if (cur == key) {
                done = true;
            } else if (cur == kEmpty) {
                const uint64_t prev = atomicCAS((unsigned long long*)&A.table[h], (unsigned long long)kEmpty,
                                                (unsigned long long)key);
                if (prev == kEmpty || prev == key) done = true;
                else h = (h + 1) & (A.cap - 1);
            } else {
                h = (h + 1) & (A.cap - 1);
            }
        }
        if (!done) ++fails;
    }
    if (mine) atomicAdd(&A.counters[0], mine);
    if (fails) atomicAdd(&A.counters[1], fails);
}

__global__ void oct_compact_kernel(const uint64_t* table, uint64_t cap, uint64_t* out, unsigned long long* n)
{
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < cap; k += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t v = table[k];
        if (v != kEmpty) out[atomicAdd(n, 1ull)] = v;
    }
}

// ---- host set operations on sorted Morton keys of one level
using Keys = std::vector<uint64_t>;

void sort_unique(Keys& k)
{
    std::sort(k.begin(), k.end());
    k.erase(std::unique(k.begin(), k.end()), k.end());
}

Keys dilate(const Keys& s, int64_t nbr)
{
    Keys o;
    o.reserve(s.size() * 27);
    for (uint64_t key : s) {
        const int64_t x = (int64_t)compact3(key), y = (int64_t)compact3(key >> 1), z = (int64_t)compact3(key >> 2);
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int64_t a = x + dx, b = y + dy, c = z + dz;
                    if (a < 0 || b < 0 || c < 0 || a >= nbr || b >= nbr || c >= nbr) continue;
                    o.push_back(morton3((uint64_t)a, (uint64_t)b, (uint64_t)c));
                }
    }
    sort_unique(o);
    return o;
}

void decode(const Keys& k, std::vector<int32_t>& out)
{
    out.resize(3 * k.size());
    for (size_t i = 0; i < k.size(); ++i) {
        out[3 * i] = (int32_t)compact3(k[i]);
        out[3 * i + 1] = (int32_t)compact3(k[i] >> 1);
        out[3 * i + 2] = (int32_t)compact3(k[i] >> 2);
    }
}

struct DevBuf {
    void* p = nullptr;
    ~DevBuf()
    {
        if (p) cudaFree(p);
    }
};

}  // namespace

extern "C" {

tgv_status tgv_octree_build(const tgv_octree_cfg* cfg, const tgv_camera* cams, int32_t nmaps, const float* depth_dev,
                            int64_t pitch_elems, int64_t map_stride_elems, void* stream, tgv_octree** out)
{
    if (!out) return TGV_ERR_INVALID_ARG;
    *out = nullptr;
    if (!cfg || nmaps < 0 || (nmaps > 0 && (!cams || !depth_dev))) return TGV_ERR_INVALID_ARG;
    if (!(cfg->root_edge > 0.0) || cfg->depth_min < 3 || cfg->depth_max < cfg->depth_min || cfg->depth_max > 21 ||
        cfg->band < 0 || cfg->band > 8)
        return TGV_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if (!isfinite(cfg->root_min[a])) return TGV_ERR_INVALID_ARG;
    const int W = nmaps > 0 ? cams[0].width : 1, H = nmaps > 0 ? cams[0].height : 1;
    if (W <= 0 || H <= 0 || W > 32768 || H > 32768 || (nmaps > 0 && pitch_elems < W)) return TGV_ERR_INVALID_ARG;
    if (nmaps > 1 && map_stride_elems < pitch_elems * H) return TGV_ERR_INVALID_ARG;
    for (int m = 0; m < nmaps; ++m) {
        const tgv_camera& c = cams[m];
        if (c.width != W || c.height != H) return TGV_ERR_INVALID_ARG;
        if (c.model != TGV_PINHOLE) return TGV_ERR_UNSUPPORTED;
        bool ok = isfinite(c.fx) && isfinite(c.fy) && isfinite(c.cx) && isfinite(c.cy) && c.fx > 0 && c.fy > 0;
        for (int k = 0; k < 9; ++k) ok = ok && isfinite(c.R[k]);
        for (int k = 0; k < 3; ++k) ok = ok && isfinite(c.C[k]);
        if (!ok) return TGV_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return TGV_ERR_CUDA;
    const int nlev = cfg->depth_max - cfg->depth_min + 1;
    const int batch = std::min(nmaps > 0 ? nmaps : 1, 8);
    const int64_t px = (int64_t)W * H;
    DevBuf X, table, cnt, uniq;
    if (cudaMalloc(&X.p, sizeof(float4) * (size_t)(px * batch)) != cudaSuccess ||
        cudaMalloc(&cnt.p, 2 * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        return TGV_ERR_OUT_OF_MEMORY;
    }
    uint64_t cap = (uint64_t)1 << 20;
    Keys keys;
    unsigned long long hc[2] = {0, 0};
    for (int attempt = 0; attempt < 6; ++attempt) {
        if (table.p) cudaFree(table.p);
        table.p = nullptr;
        if (cudaMalloc(&table.p, sizeof(uint64_t) * cap) != cudaSuccess) {
            cudaGetLastError();
            return TGV_ERR_OUT_OF_MEMORY;
        }
        e = cudaMemsetAsync(table.p, 0xff, sizeof(uint64_t) * cap, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(cnt.p, 0, 2 * sizeof(unsigned long long), s);
        for (int m0 = 0; e == cudaSuccess && m0 < nmaps; m0 += batch) {
            OctArgs A;
            A.nmaps = std::min(batch, nmaps - m0);
            A.depth = depth_dev + (int64_t)m0 * map_stride_elems;
            A.pitch = pitch_elems;
            A.stride = map_stride_elems;
            A.W = W;
            A.H = H;
            for (int m = 0; m < A.nmaps; ++m) {
                const tgv_camera& c = cams[m0 + m];
                OctCam& g = A.cam[m];
                g.fx = (float)c.fx;
                g.fy = (float)c.fy;
                g.cx = (float)c.cx;
                g.cy = (float)c.cy;
                for (int k = 0; k < 9; ++k) g.R[k] = (float)c.R[k];
                for (int k = 0; k < 3; ++k) g.C[k] = (float)c.C[k];
            }
            A.X = (float4*)X.p;
            for (int a = 0; a < 3; ++a) A.m[a] = (float)cfg->root_min[a];
            A.E = (float)cfg->root_edge;
            A.rroot = A.E * 0.5f;  // exact
            A.dmin = cfg->depth_min;
            A.dmax = cfg->depth_max;
            A.table = (uint64_t*)table.p;
            A.cap = cap;
            A.counters = (unsigned long long*)cnt.p;
            const int64_t n = px * A.nmaps;
            const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 16);
            oct_unproject_kernel<<<grid, 256, 0, s>>>(A);
            oct_key_kernel<<<grid, 256, 0, s>>>(A);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(hc, cnt.p, sizeof(hc), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return TGV_ERR_CUDA;
        if (hc[1] == 0) break;
        cap <<= 2;  // a probe sequence ran out: retry with a table four times larger
        if (attempt == 5) return TGV_ERR_BUDGET;
    }
    // unique keys to the host
    unsigned long long nu = 0;
    if (cudaMalloc(&uniq.p, sizeof(uint64_t) * cap) != cudaSuccess) {
        cudaGetLastError();
        return TGV_ERR_OUT_OF_MEMORY;
    }
    e = cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) {
        oct_compact_kernel<<<(unsigned)std::min<uint64_t>((cap + 255) / 256, (uint64_t)sms * 16), 256, 0, s>>>(
            (const uint64_t*)table.p, cap, (uint64_t*)uniq.p, (unsigned long long*)cnt.p);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nu, cnt.p, sizeof(nu), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) {
        keys.resize(nu);
        if (nu) e = cudaMemcpy(keys.data(), uniq.p, sizeof(uint64_t) * nu, cudaMemcpyDeviceToHost);
    }
    if (e != cudaSuccess) return TGV_ERR_CUDA;
    // levels
    std::vector<Keys> act(nlev);
    for (uint64_t k : keys) act[k >> 57].push_back(k & ((((uint64_t)1) << 57) - 1));
    auto per_axis = [&](int l) -> int64_t { return std::max<int64_t>(((int64_t)1 << (cfg->depth_min + l)) >> 3, 1); };
    for (int l = 0; l < nlev; ++l) {
        sort_unique(act[l]);
        for (int b = 0; b < cfg->band; ++b) act[l] = dilate(act[l], per_axis(l));
    }
    for (int l = nlev - 1; l >= 1; --l) {
        Keys par;
        par.reserve(act[l].size());
        for (uint64_t k : act[l]) par.push_back(morton3(compact3(k) >> 1, compact3(k >> 1) >> 1, compact3(k >> 2) >> 1));
        sort_unique(par);
        Keys dl = dilate(par, per_axis(l - 1));
        act[l - 1].insert(act[l - 1].end(), dl.begin(), dl.end());
        sort_unique(act[l - 1]);
    }
    tgv_octree* o = new (std::nothrow) tgv_octree();
    if (!o) return TGV_ERR_OUT_OF_MEMORY;
    o->samples = (int64_t)hc[0];
    o->levels.resize(nlev);
    for (int l = 0; l < nlev; ++l) {
        Keys frz;
        if (l > 0) {
            Keys dl = dilate(act[l], per_axis(l));
            std::set_difference(dl.begin(), dl.end(), act[l].begin(), act[l].end(), std::back_inserter(frz));
        }
        decode(act[l], o->levels[l].active);
        decode(frz, o->levels[l].frozen);
        const double h = cfg->root_edge / (double)((int64_t)1 << (cfg->depth_min + l));
        for (int a = 0; a < 3; ++a) o->levels[l].origin[a] = cfg->root_min[a];
        o->levels[l].h = h;
    }
    *out = o;
    return TGV_OK;
}

tgv_status tgv_octree_level(const tgv_octree* o, int32_t level, int64_t* nactive, int64_t* nfrozen, double* origin,
                            double* h)
{
    if (!o || level < 0 || level >= (int32_t)o->levels.size()) return TGV_ERR_INVALID_ARG;
    const tgv_octree::Level& L = o->levels[level];
    if (nactive) *nactive = (int64_t)L.active.size() / 3;
    if (nfrozen) *nfrozen = (int64_t)L.frozen.size() / 3;
    if (origin)
        for (int a = 0; a < 3; ++a) origin[a] = L.origin[a];
    if (h) *h = L.h;
    return TGV_OK;
}

tgv_status tgv_octree_bricks(const tgv_octree* o, int32_t level, int32_t* active, int32_t* frozen)
{
    if (!o || level < 0 || level >= (int32_t)o->levels.size()) return TGV_ERR_INVALID_ARG;
    const tgv_octree::Level& L = o->levels[level];
    if ((!L.active.empty() && !active) || (!L.frozen.empty() && !frozen)) return TGV_ERR_INVALID_ARG;
    std::copy(L.active.begin(), L.active.end(), active);
    std::copy(L.frozen.begin(), L.frozen.end(), frozen);
    return TGV_OK;
}

int32_t tgv_octree_levels(const tgv_octree* o) { return o ? (int32_t)o->levels.size() : 0; }

int64_t tgv_octree_samples(const tgv_octree* o) { return o ? o->samples : 0; }

void tgv_octree_destroy(tgv_octree* o) { delete o; }

}  // extern "C"
