// Brick domains from depth maps (Sec. 3.3 Eq. 4, Sec. 4.1-4.2), in memory.
//
// Every valid pixel is a point sample X (a pinhole map's z-depth, or a spherical
// map's range along the pixel's azimuth and elevation, unprojected) with radius
// r = half the mean distance to the points of its valid 4-neighbours (left,
// right, up, down).  Eq. 4 puts the sample in the cube
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
// detected and the build retried with a larger one).  The levels are formed from
// the unique keys in a second device hash set, with no host pass over the keys:
// dilation by `band` rings of 26-neighbours (all levels at once), the 2:1 balance
// (finest first, level l-1 gains the parents b >> 1 of level l's bricks dilated
// once, so every finer level is wrapped by a shell of the next coarser one), and
// the frozen shell of each level above the coarsest (26-neighbours of its active
// bricks that are not active) in a third set.  A stable LSD radix sort on the
// device orders both sets by (level, Morton code); the host only splits the
// sorted keys into levels and decodes the coordinates.
#include <math.h>

#include <algorithm>
#include <vector>

#include "tgv_internal.cuh"
#include "tgv_zorder.cuh"
#include "tgv_nvtx.h"

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

// splitmix64 finaliser (Steele, Lea, Flood 2014) as the hash of a key
__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

constexpr int kLevelShift = 57;
constexpr uint64_t kMortonMask = ((uint64_t)1 << kLevelShift) - 1;

// ---- device hash sets of 64-bit keys (open addressing, linear probing bounded by
// kMaxProbe; a key never moves once written, so a slot reads either empty or final)
__device__ __forceinline__ bool set_insert(uint64_t* table, uint64_t cap, uint64_t key)
{
    uint64_t h = mix64(key) & (cap - 1);
    for (int probe = 0; probe < kMaxProbe; ++probe) {
        const uint64_t cur = table[h];
        if (cur == key) return true;
        if (cur == kEmpty) {
            const uint64_t prev = atomicCAS((unsigned long long*)&table[h], (unsigned long long)kEmpty,
                                            (unsigned long long)key);
            if (prev == kEmpty || prev == key) return true;
        }
        h = (h + 1) & (cap - 1);
    }
    return false;
}

// membership in a set that no thread modifies meanwhile: every key present sits
// within kMaxProbe slots of its home (its insertion reported failure otherwise)
__device__ __forceinline__ bool set_contains(const uint64_t* table, uint64_t cap, uint64_t key)
{
    uint64_t h = mix64(key) & (cap - 1);
    for (int probe = 0; probe < kMaxProbe; ++probe) {
        const uint64_t cur = table[h];
        if (cur == key) return true;
        if (cur == kEmpty) return false;
        h = (h + 1) & (cap - 1);
    }
    return false;
}

struct OctCam {
    float fx, fy, cx, cy, R[9], C[3];
    int spherical;
};

// sin and cos of x in FP32 (|x| <= 4), one rounding per operation: Cody-Waite
// reduction by pi/2 (k = nearest integer to x 2/pi; r = x - k pi/2 in two fused
// multiply-adds, pi/2 split into a float head and tail), the Taylor polynomials of
// sin (to r^9) and cos (to r^10) on |r| <= pi/4 by Horner's rule in fused
// multiply-adds (truncation below 2e-9), then the quadrant k mod 4.  The oracle
// evaluates the same steps, so spherical samples unproject bit for bit alike.
__device__ __forceinline__ void sincos_tay(float x, float* s, float* c)
{
    const float two_over_pi = (float)(2.0 / 3.14159265358979323846);
    const float p1 = (float)(3.14159265358979323846 / 2.0);
    const float p2 = (float)(3.14159265358979323846 / 2.0 - (double)(float)(3.14159265358979323846 / 2.0));
    const float kf = rintf(__fmul_rn(x, two_over_pi));
    float r = __fmaf_rn(-kf, p1, x);
    r = __fmaf_rn(-kf, p2, r);
    const float r2 = __fmul_rn(r, r);
    float ps = __fmaf_rn(r2, (float)(1.0 / 362880.0), (float)(-1.0 / 5040.0));
    ps = __fmaf_rn(ps, r2, (float)(1.0 / 120.0));
    ps = __fmaf_rn(ps, r2, (float)(-1.0 / 6.0));
    const float sr = __fmaf_rn(__fmul_rn(r2, r), ps, r);
    float pc = __fmaf_rn(r2, (float)(-1.0 / 3628800.0), (float)(1.0 / 40320.0));
    pc = __fmaf_rn(pc, r2, (float)(-1.0 / 720.0));
    pc = __fmaf_rn(pc, r2, (float)(1.0 / 24.0));
    pc = __fmaf_rn(pc, r2, -0.5f);
    const float cr = __fmaf_rn(pc, r2, 1.0f);
    switch ((int)kf & 3) {
    case 0: *s = sr; *c = cr; break;
    case 1: *s = cr; *c = -sr; break;
    case 2: *s = -sr; *c = -cr; break;
    default: *s = -cr; *c = sr; break;
    }
}

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
            float pc0, pc1, pc2;
            if (c.spherical) {  // a LIDAR scan: z is the range along the pixel's direction
                float sp, cp, st, ct;
                sincos_tay(__fdiv_rn(__fsub_rn(__fadd_rn(__int2float_rn(i), 0.5f), c.cx), c.fx), &sp, &cp);
                sincos_tay(__fdiv_rn(__fsub_rn(c.cy, __fadd_rn(__int2float_rn(j), 0.5f)), c.fy), &st, &ct);
                const float rc = __fmul_rn(z, ct);
                pc0 = __fmul_rn(rc, cp);
                pc1 = __fmul_rn(rc, sp);
                pc2 = __fmul_rn(z, st);
            } else {
                pc0 = __fmul_rn(__fdiv_rn(__fsub_rn(__fadd_rn(__int2float_rn(i), 0.5f), c.cx), c.fx), z);
                pc1 = __fmul_rn(__fdiv_rn(__fsub_rn(__fadd_rn(__int2float_rn(j), 0.5f), c.cy), c.fy), z);
                pc2 = z;
            }
            float x[3];
            for (int a = 0; a < 3; ++a) {
                float s = __fadd_rn(__fmul_rn(c.R[a], pc0), __fmul_rn(c.R[3 + a], pc1));
                s = __fadd_rn(s, __fmul_rn(c.R[6 + a], pc2));
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
        const uint64_t key = ((uint64_t)(d - A.dmin) << kLevelShift) | morton3(q[0] >> 3, q[1] >> 3, q[2] >> 3);
        if (!set_insert(A.table, A.cap, key)) ++fails;
    }
    if (mine) atomicAdd(&A.counters[0], mine);
    if (fails) atomicAdd(&A.counters[1], fails);
}

// the keys of a set (of one level, or all with level < 0) to a list; *n counts them
__global__ void oct_compact_kernel(const uint64_t* table, uint64_t cap, int level, uint64_t* out,
                                   unsigned long long* n)
{
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < cap; k += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t v = table[k];
        if (v != kEmpty && (level < 0 || (int)(v >> kLevelShift) == level)) out[atomicAdd(n, 1ull)] = v;
    }
}

struct LevelDims {
    int64_t per_axis[32];  // bricks per axis of each level
};

enum NeighbourMode { kSelf = 0, kRing = 1, kParentRing = 2, kShell = 3 };

// For each key of `list` (*n of them), inserts into `dst`:
//   kSelf        the key itself;
//   kRing        its 27-neighbourhood (itself included) at its level;
//   kParentRing  the 27-neighbourhood of its parent b >> 1 one level coarser;
//   kShell       its 26 neighbours that `act` does not hold (levels above 0 only).
// Neighbours outside the level's cube are dropped.  Failed insertions are counted.
__global__ void oct_neighbour_kernel(const uint64_t* list, const unsigned long long* n, uint64_t* dst,
                                     uint64_t cap, const uint64_t* act, uint64_t act_cap, const LevelDims D,
                                     int mode, unsigned long long* fails)
{
    const uint64_t count = *n;
    unsigned long long bad = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t key = list[i];
        int l = (int)(key >> kLevelShift);
        if (mode == kSelf) {
            if (!set_insert(dst, cap, key)) ++bad;
            continue;
        }
        const uint64_t m = key & kMortonMask;
        int64_t x = (int64_t)compact3(m), y = (int64_t)compact3(m >> 1), z = (int64_t)compact3(m >> 2);
        if (mode == kParentRing) {
            if (l == 0) continue;
            --l;
            x >>= 1;
            y >>= 1;
            z >>= 1;
        }
        if (mode == kShell && l == 0) continue;
        const int64_t P = D.per_axis[l];
        const uint64_t tag = (uint64_t)l << kLevelShift;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    if (mode == kShell && dx == 0 && dy == 0 && dz == 0) continue;
                    const int64_t a = x + dx, b = y + dy, c = z + dz;
                    if (a < 0 || b < 0 || c < 0 || a >= P || b >= P || c >= P) continue;
                    const uint64_t nk = tag | morton3((uint64_t)a, (uint64_t)b, (uint64_t)c);
                    if (mode == kShell && set_contains(act, act_cap, nk)) continue;
                    if (!set_insert(dst, cap, nk)) ++bad;
                }
    }
    if (bad) atomicAdd(fails, bad);
}

// ---- stable LSD radix sort of 64-bit keys, 8-bit digits, tiles of 1024 keys
constexpr int kRsThreads = 256, kRsTile = 1024;

// digit counts of each tile, digit-major: hist[digit * tiles + tile]
__global__ void __launch_bounds__(kRsThreads) rs_hist_kernel(const uint64_t* keys, int64_t n, int shift,
                                                               uint32_t* hist, int64_t tiles)
{
    __shared__ uint32_t s[256];
    s[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
    for (int k = threadIdx.x; k < kRsTile; k += kRsThreads) {
        const int64_t i = base + k;
        if (i < n) atomicAdd(&s[(keys[i] >> shift) & 0xff], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * tiles + blockIdx.x] = s[threadIdx.x];
}

// exclusive prefix sum of m counts in place, by one block of 1024 threads, starting
// from `carry`
__device__ void block_exclusive_scan(uint32_t* a, int64_t m, uint32_t carry)
{
    __shared__ uint32_t wsum[32];
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    for (int64_t base = 0; base < m; base += 1024) {
        const int64_t i = base + t;
        const uint32_t v = i < m ? a[i] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        if (w == 0) {
            uint32_t s = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            wsum[lane] = s;
        }
        __syncthreads();
        if (i < m) a[i] = carry + (w ? wsum[w - 1] : 0u) + x - v;
        carry += wsum[31];
        __syncthreads();  // wsum is rewritten by the next chunk
    }
}

__global__ void __launch_bounds__(1024) rs_scan_kernel(uint32_t* a, int64_t m) { block_exclusive_scan(a, m, 0u); }

// Larger count arrays: segments of kRsSeg counts, one block each -- the segment sums,
// their scan (one block), then each segment's scan from its prefix.
constexpr int64_t kRsSeg = 8192;

__global__ void __launch_bounds__(1024) rs_seg_sum_kernel(const uint32_t* a, int64_t m, uint32_t* sums)
{
    __shared__ uint32_t wsum[32];
    const int64_t base = (int64_t)blockIdx.x * kRsSeg;
    uint32_t x = 0;
    for (int64_t i = base + threadIdx.x; i < base + kRsSeg && i < m; i += 1024) x += a[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
        x = wsum[threadIdx.x];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (threadIdx.x == 0) sums[blockIdx.x] = x;
    }
}

__global__ void __launch_bounds__(1024) rs_seg_scan_kernel(uint32_t* a, int64_t m, const uint32_t* sums)
{
    const int64_t base = (int64_t)blockIdx.x * kRsSeg;
    block_exclusive_scan(a + base, m - base < kRsSeg ? m - base : kRsSeg, sums[blockIdx.x]);
}

// each tile's keys to their slots: the tile's first slot of the digit plus the key's
// rank among the tile's earlier keys of that digit (ranks in index order: stable)
__global__ void __launch_bounds__(kRsThreads) rs_scatter_kernel(const uint64_t* in, uint64_t* out, int64_t n,
                                                                  int shift, const uint32_t* offs, int64_t tiles)
{
    __shared__ uint32_t s_run[256];
    __shared__ uint32_t s_cnt[kRsThreads / 32][256];
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    s_run[t] = offs[(int64_t)t * tiles + blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
    for (int r = 0; r < kRsTile / kRsThreads; ++r) {
#pragma unroll
        for (int k = 0; k < kRsThreads / 32; ++k) s_cnt[k][t] = 0;
        __syncthreads();
        const int64_t i = base + r * kRsThreads + t;
        const bool valid = i < n;
        const uint64_t key = valid ? in[i] : 0;
        const uint32_t dg = valid ? (uint32_t)((key >> shift) & 0xff) : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, dg);
        const unsigned rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank == 0) s_cnt[w][dg] = __popc(peers);
        __syncthreads();
        uint32_t acc = 0;  // digit t: counts of the earlier warps
#pragma unroll
        for (int k = 0; k < kRsThreads / 32; ++k) {
            const uint32_t c = s_cnt[k][t];
            s_cnt[k][t] = acc;
            acc += c;
        }
        __syncthreads();
        if (valid) out[s_run[dg] + s_cnt[w][dg] + rank] = key;
        __syncthreads();
        s_run[t] += acc;
    }
}

int64_t radix_hist_words(int64_t n)
{
    const int64_t m = 256 * std::max<int64_t>((n + kRsTile - 1) / kRsTile, 1);
    return m + (m + kRsSeg - 1) / kRsSeg + 1;
}

// sorts n keys by the 8-bit digits at `shifts` (least significant first); `tmp`
// holds n keys, `hist` radix_hist_words(n) counts; adds its launches to *launches.
// With `result` the sorted keys stay in whichever of keys / tmp the last pass wrote and
// *result points there; without it they are copied back into keys.
cudaError_t radix_sort(uint64_t* keys, uint64_t* tmp, uint32_t* hist, int64_t n, const std::vector<int>& shifts,
                       cudaStream_t s, int64_t* launches = nullptr, uint64_t** result = nullptr)
{
    if (result) *result = keys;
    if (n <= 1) return cudaSuccess;
    const int64_t tiles = (n + kRsTile - 1) / kRsTile, m = 256 * tiles, segs = (m + kRsSeg - 1) / kRsSeg;
    uint64_t *a = keys, *b = tmp;
    for (int sh : shifts) {
        rs_hist_kernel<<<(unsigned)tiles, kRsThreads, 0, s>>>(a, n, sh, hist, tiles);
        if (segs == 1) {
            rs_scan_kernel<<<1, 1024, 0, s>>>(hist, m);
        } else {
            rs_seg_sum_kernel<<<(unsigned)segs, 1024, 0, s>>>(hist, m, hist + m);
            rs_scan_kernel<<<1, 1024, 0, s>>>(hist + m, segs);
            rs_seg_scan_kernel<<<(unsigned)segs, 1024, 0, s>>>(hist, m, hist + m);
        }
        rs_scatter_kernel<<<(unsigned)tiles, kRsThreads, 0, s>>>(a, b, n, sh, hist, tiles);
        if (launches) *launches += segs == 1 ? 3 : 5;
        std::swap(a, b);
    }
    if (result) {
        *result = a;
        return cudaGetLastError();
    }
    if (a != keys) return cudaMemcpyAsync(keys, a, sizeof(uint64_t) * (size_t)n, cudaMemcpyDeviceToDevice, s);
    return cudaGetLastError();
}

void decode(const uint64_t* k, size_t n, std::vector<int32_t>& out)
{
    out.resize(3 * n);
    for (size_t i = 0; i < n; ++i) {
        const uint64_t m = k[i] & kMortonMask;
        out[3 * i] = (int32_t)compact3(m);
        out[3 * i + 1] = (int32_t)compact3(m >> 1);
        out[3 * i + 2] = (int32_t)compact3(m >> 2);
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

cudaError_t tgv_radix_sort_u64(uint64_t* keys, uint64_t* tmp, uint32_t* hist, int64_t n, int lo_bit, int nbits,
                               cudaStream_t s, int64_t* launches, uint64_t** result)
{
    std::vector<int> shifts;
    for (int b = 0; b < nbits; b += 8) shifts.push_back(lo_bit + b);
    return radix_sort(keys, tmp, hist, n, shifts, s, launches, result);
}

int64_t tgv_radix_hist_words(int64_t n) { return radix_hist_words(n); }

extern "C" {

tgv_status tgv_octree_build(const tgv_octree_cfg* cfg, const tgv_camera* cams, int32_t nmaps, const float* depth_dev,
                            int64_t pitch_elems, int64_t map_stride_elems, void* stream, tgv_octree** out)
{
    TgvNvtxRange nvtx_range_("tgv_octree_build");
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
        if (c.model != TGV_PINHOLE && c.model != TGV_SPHERICAL) return TGV_ERR_INVALID_ARG;
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
                g.spherical = c.model == TGV_SPHERICAL;
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
    // unique sample keys to a list on the device
    unsigned long long nu = 0;
    if (cudaMalloc(&uniq.p, sizeof(uint64_t) * cap) != cudaSuccess) {
        cudaGetLastError();
        return TGV_ERR_OUT_OF_MEMORY;
    }
    const unsigned sgrid = (unsigned)sms * 8;
    auto compact = [&](const void* tab, uint64_t c, int level, void* list, unsigned long long* n) -> cudaError_t {
        cudaError_t r = cudaMemsetAsync(n, 0, sizeof(unsigned long long), s);
        if (r != cudaSuccess) return r;
        oct_compact_kernel<<<(unsigned)std::min<uint64_t>((c + 255) / 256, (uint64_t)sms * 16), 256, 0, s>>>(
            (const uint64_t*)tab, c, level, (uint64_t*)list, n);
        return cudaGetLastError();
    };
    unsigned long long* dcnt = (unsigned long long*)cnt.p;
    e = compact(table.p, cap, -1, uniq.p, dcnt);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nu, dcnt, sizeof(nu), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return TGV_ERR_CUDA;
    cudaFree(table.p);
    table.p = nullptr;

    LevelDims D;
    for (int l = 0; l < 32; ++l)
        D.per_axis[l] = l < nlev ? std::max<int64_t>(((int64_t)1 << (cfg->depth_min + l)) >> 3, 1) : 1;
    // level sets: active (act) and frozen shells (frz), with their key lists
    DevBuf act, frz, lst, lst2, tmp, hist, sc;
    unsigned long long hs[3] = {0, 0, 0};  // failed insertions, active keys, frozen keys
    if (cudaMalloc(&sc.p, 3 * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        return TGV_ERR_OUT_OF_MEMORY;
    }
    unsigned long long* dsc = (unsigned long long*)sc.p;
    // slots: twice the sample bricks grown by the band (a layer thickens by 2 band + 1
    // bricks, a line by its square), at least 2^20; a table that fills is redone larger
    const uint64_t grow = std::min<uint64_t>((uint64_t)(2 * cfg->band + 1) * (2 * cfg->band + 1), 32);
    uint64_t cap2 = (uint64_t)1 << 20;
    while (cap2 < 2 * grow * (uint64_t)nu) cap2 <<= 1;
    for (int attempt = 0; nu > 0; ++attempt) {
        for (DevBuf* b : {&act, &frz, &lst, &lst2, &tmp, &hist}) {
            if (b->p) cudaFree(b->p);
            b->p = nullptr;
        }
        const size_t kb = sizeof(uint64_t) * cap2;
        if (cudaMalloc(&act.p, kb) != cudaSuccess || cudaMalloc(&frz.p, kb) != cudaSuccess ||
            cudaMalloc(&lst.p, kb) != cudaSuccess || cudaMalloc(&lst2.p, kb) != cudaSuccess ||
            cudaMalloc(&tmp.p, kb) != cudaSuccess ||
            cudaMalloc(&hist.p, sizeof(uint32_t) * (size_t)radix_hist_words(cap2)) != cudaSuccess) {
            cudaGetLastError();
            return TGV_ERR_OUT_OF_MEMORY;
        }
        uint64_t *A = (uint64_t*)act.p, *F = (uint64_t*)frz.p, *L1 = (uint64_t*)lst.p, *L2 = (uint64_t*)lst2.p;
        e = cudaMemsetAsync(A, 0xff, kb, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(F, 0xff, kb, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(dsc, 0, 3 * sizeof(unsigned long long), s);
        auto expand = [&](const uint64_t* list, const unsigned long long* n, uint64_t* dst, const uint64_t* in,
                          int mode) {
            if (e != cudaSuccess) return;
            oct_neighbour_kernel<<<sgrid, 256, 0, s>>>(list, n, dst, cap2, in, cap2, D, mode, dsc);
            e = cudaGetLastError();
        };
        auto list_of = [&](const uint64_t* tab, int level, uint64_t* list, unsigned long long* n) {
            if (e == cudaSuccess) e = compact(tab, cap2, level, list, n);
        };
        // the sample bricks, then `band` rings of neighbours on every level at once
        expand((const uint64_t*)uniq.p, dcnt, A, nullptr, kSelf);
        for (int b = 0; b < cfg->band; ++b) {
            list_of(A, -1, L1, dsc + 1);
            expand(L1, dsc + 1, A, nullptr, kRing);
        }
        // 2:1 balance, finest level first (level l-1 sees level l's final bricks)
        for (int l = nlev - 1; l >= 1; --l) {
            list_of(A, l, L1, dsc + 1);
            expand(L1, dsc + 1, A, nullptr, kParentRing);
        }
        // frozen shells from the final active bricks of all levels
        list_of(A, -1, L1, dsc + 1);
        expand(L1, dsc + 1, F, A, kShell);
        list_of(F, -1, L2, dsc + 2);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hs, dsc, sizeof(hs), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return TGV_ERR_CUDA;
        if (hs[0] == 0) break;
        if (attempt == 5) return TGV_ERR_BUDGET;
        cap2 <<= 2;  // a probe sequence ran out: redo the level sets in a larger table
    }
    // order both sets by (level, Morton code): the Morton digits of the finest level,
    // then the level digit
    std::vector<int> shifts;
    for (int sh = 0; sh < 3 * (cfg->depth_max - 3); sh += 8) shifts.push_back(sh);
    shifts.push_back(kLevelShift);
    std::vector<uint64_t> ka(hs[1]), kf(hs[2]);
    if (nu > 0) {
        e = radix_sort((uint64_t*)lst.p, (uint64_t*)tmp.p, (uint32_t*)hist.p, (int64_t)hs[1], shifts, s);
        if (e == cudaSuccess)
            e = radix_sort((uint64_t*)lst2.p, (uint64_t*)tmp.p, (uint32_t*)hist.p, (int64_t)hs[2], shifts, s);
        if (e == cudaSuccess && hs[1])
            e = cudaMemcpyAsync(ka.data(), lst.p, sizeof(uint64_t) * hs[1], cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && hs[2])
            e = cudaMemcpyAsync(kf.data(), lst2.p, sizeof(uint64_t) * hs[2], cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return TGV_ERR_CUDA;
    }
    tgv_octree* o = new (std::nothrow) tgv_octree();
    if (!o) return TGV_ERR_OUT_OF_MEMORY;
    o->samples = (int64_t)hc[0];
    o->levels.resize(nlev);
    // split the sorted keys into their levels
    auto split = [&](const std::vector<uint64_t>& k, bool frozen) {
        size_t i = 0;
        for (int l = 0; l < nlev; ++l) {
            size_t j = i;
            while (j < k.size() && (int)(k[j] >> kLevelShift) == l) ++j;
            decode(k.data() + i, j - i, frozen ? o->levels[l].frozen : o->levels[l].active);
            i = j;
        }
    };
    split(ka, false);
    split(kf, true);
    for (int l = 0; l < nlev; ++l) {
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
