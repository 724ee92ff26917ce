// Joint solve of all levels on their composite grid (Sec. 3.3: a cube of a
// 2:1-balanced octree has up to four neighbours over a face; Eq. 2-3, Sec. 3.2).
//
// Leaves: voxels of level l in an active brick whose 8 children (level l+1) are
// not in an active brick -- children of one voxel lie in one finer brick.  Every
// difference is a unit index step, as on a single level.  For leaf x and axis a
// the +a neighbours are the same-level leaf x + e_a; else, when level l has no
// voxel there, the coarser leaf that contains it; else, when that voxel is
// refined, its 4 children on the face next to x; else none (likewise -a):
//   (G_a u)(x) = mean(u over +a neighbours) - u(x)    (0 without neighbours)
//   (B_a w)(x) = w(x) - mean(w over -a neighbours)    (0 without neighbours)
//   E(v)_ab = (B_a v_b + B_b v_a) / 2,  div1 = -sum_a G_a^T,  (div2 q)_b = -sum_a B_a^T q_ab.
// The adjoints are exact: each leaf keeps, per axis, the leaves whose +a (-a)
// neighbour lists contain it with their weight 1 / (list length).  On a single
// level all of this is the iteration of tgv_iter_kernel without frozen bricks.
//
// State per leaf in FP32 (u, ubar, v, vbar, p, q and the packed histogram of its
// level).  Regular leaves (one same-level neighbour or none per side) carry six
// neighbour ids; leaves at 2:1 faces carry the full lists.  One iteration = a dual kernel (p, q from ubar, vbar and the neighbour
// lists) and a primal kernel (divergences through the reverse lists, prox,
// clamp, v update, over-relaxation), one thread per leaf.
//
// Treetop (Sec. 4.3): the leaves are the octree's leaf cubes.  In Z-order (Morton
// order of the lower corners, in finest voxel units) the cubes under a node are
// consecutive; the treetop keeps splitting, from the root down, every node that
// holds N or more cubes, and its leaf nodes (parts) each hold fewer than N.
#include <math.h>

#include <algorithm>
#include <memory>
#include <vector>

#include "tgv_internal.cuh"
#include "tgv_zorder.cuh"
#include "tgv_nvtx.h"

struct tgv_composite {
    tgv_domain* d = nullptr;
    int64_t n = 0;
    std::vector<int64_t> level_first;             // first leaf of each level (and the total)
    int32_t* slot = nullptr;                      // [n]: slot (brick * 512 + local) of each leaf in its level
    float *u = nullptr, *ubar = nullptr, *v = nullptr, *vbar = nullptr, *p = nullptr, *q = nullptr;
    uint32_t* hist = nullptr;                     // [n][npairs]
    int32_t* nb6 = nullptr;                       // [n][6]: +x +y +z -x -y -z neighbour of a regular leaf
    int32_t* lists = nullptr;                     // [irregular][4 kinds][3 axes][4]: fwd, bwd, rev fwd, rev bwd
    int64_t nirr = 0;
    int64_t launches = 0;
    // treetop of the last tgv_composite_treetop call (Sec. 4.3)
    std::vector<int32_t> tt_depth;
    std::vector<uint64_t> tt_code;
    std::vector<int64_t> tt_first, tt_last;
    int32_t* tt_part = nullptr;                   // [n]: treetop part of each leaf
};

namespace {

constexpr int kList = 4;
constexpr uint32_t kQuarter = 0x80000000u;  // reverse-list weight 1/4 (else 1)

struct CompArgs {
    float *u, *ubar, *v, *vbar, *p, *q;
    const uint32_t* hist;
    const int32_t* nb6;    // regular leaf: six neighbour ids (-1 none); irregular: nb6[0] = -2 - index
    const int32_t* lists;  // full lists of the irregular leaves
    int64_t n;
    int nbins, npairs, clamp_u;
    float alpha1, alpha0, tau, sigma, taulam;
    float c[TGV_MAX_BINS];
};

__device__ __forceinline__ const int32_t* list_of(const CompArgs& A, int64_t irr, int kind, int a)
{
    return A.lists + ((irr * 4 + kind) * 3 + a) * kList;
}

// Most leaves are regular: one same-level neighbour (or none) on every side,
// so their reverse lists are the mirrored neighbours with weight 1 and six ids
// describe them.  Leaves at 2:1 faces keep the full lists.
__device__ __forceinline__ void comp_dual_leaf(const CompArgs& A, const int64_t x)
{
    if (x >= A.n) return;
    const float ub = A.ubar[x];
    float vb[3], g[3], dm[3][3];
    for (int c = 0; c < 3; ++c) vb[c] = A.vbar[3 * x + c];
    const int32_t m0 = A.nb6[6 * x];
    if (m0 > -2) {
        for (int a = 0; a < 3; ++a) {
            const int32_t f = A.nb6[6 * x + a], bk = A.nb6[6 * x + 3 + a];
            g[a] = f >= 0 ? A.ubar[f] - ub : 0.0f;
            for (int c = 0; c < 3; ++c) dm[a][c] = bk >= 0 ? vb[c] - A.vbar[3 * (int64_t)bk + c] : 0.0f;
        }
    } else {
    const int64_t irr = -2 - (int64_t)m0;
    for (int a = 0; a < 3; ++a) {
        const int32_t* f = list_of(A, irr, 0, a);
        int cnt = 0;
        float s = 0.0f;
        for (int k = 0; k < kList; ++k)
            if (f[k] >= 0) {
                s += A.ubar[f[k]];
                ++cnt;
            }
        g[a] = cnt ? (cnt == 1 ? s : 0.25f * s) - ub : 0.0f;
        const int32_t* bl = list_of(A, irr, 1, a);
        float w[3] = {0.0f, 0.0f, 0.0f};
        cnt = 0;
        for (int k = 0; k < kList; ++k)
            if (bl[k] >= 0) {
                for (int c = 0; c < 3; ++c) w[c] += A.vbar[3 * (int64_t)bl[k] + c];
                ++cnt;
            }
        for (int c = 0; c < 3; ++c) dm[a][c] = cnt ? vb[c] - (cnt == 1 ? w[c] : 0.25f * w[c]) : 0.0f;
    }
    }
    float pn[3], qn[6];
    for (int c = 0; c < 3; ++c) pn[c] = A.p[3 * x + c] + A.sigma * (g[c] - vb[c]);
    const float n2 = pn[0] * pn[0] + pn[1] * pn[1] + pn[2] * pn[2];
    if (n2 > A.alpha1 * A.alpha1) {
        const float s = A.alpha1 / sqrtf(n2);
        for (int c = 0; c < 3; ++c) pn[c] *= s;
    }
    const float e[6] = {dm[0][0], dm[1][1], dm[2][2], 0.5f * (dm[0][1] + dm[1][0]), 0.5f * (dm[0][2] + dm[2][0]),
                        0.5f * (dm[1][2] + dm[2][1])};
    for (int c = 0; c < 6; ++c) qn[c] = A.q[6 * x + c] + A.sigma * e[c];
    const float q2 = qn[0] * qn[0] + qn[1] * qn[1] + qn[2] * qn[2] + 2.0f * (qn[3] * qn[3] + qn[4] * qn[4] + qn[5] * qn[5]);
    if (q2 > A.alpha0 * A.alpha0) {
        const float s = A.alpha0 / sqrtf(q2);
        for (int c = 0; c < 6; ++c) qn[c] *= s;
    }
    for (int c = 0; c < 3; ++c) A.p[3 * x + c] = pn[c];
    for (int c = 0; c < 6; ++c) A.q[6 * x + c] = qn[c];
}

__global__ void comp_dual_kernel(const CompArgs A)
{
    const int64_t x = (int64_t)blockIdx.x * (2 * blockDim.x) + threadIdx.x;
    comp_dual_leaf(A, x);
    comp_dual_leaf(A, x + blockDim.x);
}

__device__ __forceinline__ int qidx_c(int a, int b) { return a == b ? a : (a + b == 1 ? 3 : (a + b == 2 ? 4 : 5)); }

template <int NB>  // bin count (0: read at run time)
__device__ __forceinline__ void comp_primal_leaf(const CompArgs& A, const int64_t x)
{
    constexpr int NBM = NB ? NB : TGV_MAX_BINS;
    if (x >= A.n) return;
    float d1 = 0.0f, d2[3] = {0.0f, 0.0f, 0.0f};
    const int32_t m0 = A.nb6[6 * x];
    if (m0 > -2) {
        for (int a = 0; a < 3; ++a) {
            const int32_t f = A.nb6[6 * x + a], bk = A.nb6[6 * x + 3 + a];
            if (f >= 0) d1 += A.p[3 * x + a];
            if (bk >= 0) d1 -= A.p[3 * (int64_t)bk + a];
            for (int b = 0; b < 3; ++b) {
                const int qc = qidx_c(a, b);
                if (bk >= 0) d2[b] -= A.q[6 * x + qc];
                if (f >= 0) d2[b] += A.q[6 * (int64_t)f + qc];
            }
        }
    } else {
    const int64_t irr = -2 - (int64_t)m0;
    for (int a = 0; a < 3; ++a) {
        // div1 = sum_a ([x has +a neighbours] p_a(x) - sum over reverse +a list of w p_a(r))
        if (list_of(A, irr, 0, a)[0] >= 0) d1 += A.p[3 * x + a];
        const int32_t* rf = list_of(A, irr, 2, a);
        for (int k = 0; k < kList; ++k)
            if (rf[k] != -1) {
                const int64_t r = rf[k] & 0x7fffffff;
                const float w = ((uint32_t)rf[k] & kQuarter) ? 0.25f : 1.0f;
                d1 -= w * A.p[3 * r + a];
            }
        // (div2 q)_b = sum_a (-[x has -a neighbours] q_ab(x) + sum over reverse -a list of w q_ab(r))
        const bool hb = list_of(A, irr, 1, a)[0] >= 0;
        const int32_t* rb = list_of(A, irr, 3, a);
        for (int b = 0; b < 3; ++b) {
            const int qc = qidx_c(a, b);
            if (hb) d2[b] -= A.q[6 * x + qc];
            for (int k = 0; k < kList; ++k)
                if (rb[k] != -1) {
                    const int64_t r = rb[k] & 0x7fffffff;
                    const float w = ((uint32_t)rb[k] & kQuarter) ? 0.25f : 1.0f;
                    d2[b] += w * A.q[6 * r + qc];
                }
        }
    }
    }
    const float u0 = A.u[x];
    const float ut = u0 + A.tau * d1;
    // prox: generalised median = max_i min(ut - tau*lambda*W_i, c_i), c_n = +inf
    const int nbins = NB ? NB : A.nbins;
    const int npairs = NB ? (NB + 1) / 2 : A.npairs;
    uint32_t hw[(NBM + 1) / 2];
#pragma unroll
    for (int k = 0; k < (NBM + 1) / 2; ++k) hw[k] = (NB || k < npairs) ? A.hist[x * npairs + k] : 0u;
    float hs = 0.0f, hb_[NBM];
#pragma unroll
    for (int k = 0; k < NBM; ++k) {
        hb_[k] = (float)((hw[k >> 1] >> ((k & 1) * 16)) & 0xffffu);
        hs += hb_[k];
    }
    float W = -hs, un = -INFINITY;
#pragma unroll
    for (int i = 0; i < NBM; ++i) {
        if (NB || i < nbins) {
            un = fmaxf(un, fminf(ut - A.taulam * W, A.c[i]));
            W += 2.0f * hb_[i];
        }
    }
    un = fmaxf(un, ut - A.taulam * W);
    if (A.clamp_u) un = fminf(1.0f, fmaxf(-1.0f, un));
    A.u[x] = un;
    A.ubar[x] = 2.0f * un - u0;
    for (int c = 0; c < 3; ++c) {
        const float v0 = A.v[3 * x + c];
        const float v1 = v0 + A.tau * (A.p[3 * x + c] + d2[c]);
        A.v[3 * x + c] = v1;
        A.vbar[3 * x + c] = 2.0f * v1 - v0;
    }
}

// two leaves per thread (x and x + blockDim.x of the block's 2 blockDim.x leaves)
template <int NB>
__global__ void comp_primal_kernel(const CompArgs A)
{
    const int64_t x = (int64_t)blockIdx.x * (2 * blockDim.x) + threadIdx.x;
    comp_primal_leaf<NB>(A, x);
    comp_primal_leaf<NB>(A, x + blockDim.x);
}

// leaf histograms: gather the packed words of each leaf from its level
__global__ void comp_gather_hist(uint32_t* dst, const uint32_t* src, const int32_t* slot, int64_t n, int npairs)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n * npairs; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = k / npairs;
        const int j = (int)(k - x * npairs);
        const int64_t s = slot[x];
        dst[k] = src[(s / TGV_BVOX * npairs + j) * TGV_BVOX + s % TGV_BVOX];
    }
}

__global__ void comp_gather_u(float* dst, float* dst2, const float* src, const int32_t* slot, int64_t n)
{
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        const float v = src[slot[x]];
        dst[x] = v;
        dst2[x] = v;
    }
}

__global__ void comp_scatter_u(float* dst, const float* src, const int32_t* slot, int64_t n)
{
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
        dst[slot[x]] = src[x];
}

// ---- building the leaves and their lists on the device
//
// Per level a hash table maps brick coordinates to the active brick index.  A
// brick's refined octants (those whose 8^3 children form an active brick of the
// next level) give its leaf count; an exclusive scan over all bricks, level by
// level, numbers the leaves in level, brick and voxel order.  One thread per leaf
// then forms its forward and backward lists, appends itself to the reverse lists
// of the leaves it lists (compare-and-swap into the first free of four slots)
// and, after each reverse list is sorted by leaf id (the order a serial pass in
// leaf order gives), classifies it as regular or irregular.
constexpr uint64_t kNoKey = ~(uint64_t)0;
constexpr int kCoordBits = 20;  // brick coordinates lie in [-2^19, 2^19)
constexpr int kMaxProbeC = 4096;

struct CBLevel {
    const int32_t* coords;  // 3 per brick, active first
    int64_t nb;             // active bricks
    int64_t bfirst;         // first brick of the level in the global brick order
    uint64_t hoff, hcap;    // the level's slice of the hash table (cap a power of two)
    int64_t lfirst;         // first leaf of the level
};

struct CBArgs {
    CBLevel L[32];
    int nlev;
    uint64_t* hkeys;
    int32_t* hvals;
    uint32_t* base;        // [bricks]: leaf count, then (scanned) the brick's first leaf
    uint8_t* mask;         // [bricks]: octants refined by the next level
    int32_t* leaf_of;      // [bricks * 512]: leaf id of each voxel slot, -1 refined
    int32_t* slot;         // [n]: slot of each leaf in its level
    int32_t* lists;        // [n][4 kinds][3 axes][4]
    int32_t* nb6;
    int64_t n, nbt;
    unsigned int* err;     // [0] a refined voxel lacks a child, [1] more than four over a face, [2] table full
};

__device__ __forceinline__ uint64_t cb_mix(uint64_t z)
{
    // splitmix64 finaliser (Steele, Lea, Flood 2014)
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ bool cb_key(int64_t x, int64_t y, int64_t z, uint64_t& key)
{
    const int64_t B = (int64_t)1 << (kCoordBits - 1);
    if (x < -B || x >= B || y < -B || y >= B || z < -B || z >= B) return false;
    key = (uint64_t)(x + B) | ((uint64_t)(y + B) << kCoordBits) | ((uint64_t)(z + B) << (2 * kCoordBits));
    return true;
}

// active brick index of brick (x, y, z) on level l, -1 none
__device__ __forceinline__ int64_t cb_brick(const CBArgs& A, int l, int64_t x, int64_t y, int64_t z)
{
    uint64_t key;
    if (l < 0 || l >= A.nlev || !cb_key(x, y, z, key)) return -1;
    const CBLevel& L = A.L[l];
    if (L.nb == 0) return -1;
    uint64_t h = cb_mix(key) & (L.hcap - 1);
    for (int probe = 0; probe < kMaxProbeC; ++probe) {
        const uint64_t cur = A.hkeys[L.hoff + h];
        if (cur == key) return A.hvals[L.hoff + h];
        if (cur == kNoKey) return -1;
        h = (h + 1) & (L.hcap - 1);
    }
    return -1;
}

// leaf at global voxel (x, y, z) of level l: its id, -1 refined, -2 no voxel there
__device__ __forceinline__ int64_t cb_leaf(const CBArgs& A, int l, int64_t x, int64_t y, int64_t z)
{
    const int64_t b = cb_brick(A, l, x >> 3, y >> 3, z >> 3);
    if (b < 0) return -2;
    return A.leaf_of[(A.L[l].bfirst + b) * TGV_BVOX + (x & 7) + 8 * (y & 7) + 64 * (z & 7)];
}

__device__ __forceinline__ int cb_level_of_brick(const CBArgs& A, int64_t g)
{
    int l = 0;
    while (l + 1 < A.nlev && A.L[l + 1].bfirst <= g) ++l;
    return l;
}

__device__ __forceinline__ int cb_level_of_leaf(const CBArgs& A, int64_t x)
{
    int l = 0;
    while (l + 1 < A.nlev && A.L[l + 1].lfirst <= x) ++l;
    return l;
}

__global__ void cb_insert_kernel(const CBArgs A)
{
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < A.nbt; g += (int64_t)gridDim.x * blockDim.x) {
        const int l = cb_level_of_brick(A, g);
        const CBLevel& L = A.L[l];
        const int64_t b = g - L.bfirst;
        uint64_t key;
        cb_key(L.coords[3 * b], L.coords[3 * b + 1], L.coords[3 * b + 2], key);  // in range (checked at creation)
        uint64_t h = cb_mix(key) & (L.hcap - 1);
        bool done = false;
        for (int probe = 0; probe < kMaxProbeC && !done; ++probe) {
            const uint64_t prev = atomicCAS((unsigned long long*)&A.hkeys[L.hoff + h], (unsigned long long)kNoKey,
                                            (unsigned long long)key);
            if (prev == kNoKey) {
                A.hvals[L.hoff + h] = (int32_t)b;
                done = true;
            } else {
                h = (h + 1) & (L.hcap - 1);
            }
        }
        if (!done) atomicAdd(&A.err[2], 1u);
    }
}

// refined octants of each brick and its leaf count (64 per octant left)
__global__ void cb_mask_kernel(const CBArgs A)
{
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < A.nbt; g += (int64_t)gridDim.x * blockDim.x) {
        const int l = cb_level_of_brick(A, g);
        const CBLevel& L = A.L[l];
        const int64_t b = g - L.bfirst;
        const int64_t c0 = L.coords[3 * b], c1 = L.coords[3 * b + 1], c2 = L.coords[3 * b + 2];
        uint32_t m = 0;
        for (int o = 0; o < 8; ++o)
            if (cb_brick(A, l + 1, 2 * c0 + (o & 1), 2 * c1 + ((o >> 1) & 1), 2 * c2 + (o >> 2)) >= 0) m |= 1u << o;
        A.mask[g] = (uint8_t)m;
        A.base[g] = 64u * (8u - (uint32_t)__popc(m));
    }
}

// one CTA per brick: leaf ids of its voxels in voxel order
__global__ void __launch_bounds__(TGV_BVOX) cb_leaves_kernel(const CBArgs A)
{
    __shared__ uint32_t wsum[TGV_BVOX / 32];
    const int64_t g = blockIdx.x;
    const int v = threadIdx.x, w = v >> 5, lane = v & 31;
    const int o = ((v & 7) >> 2) | ((((v >> 3) & 7) >> 2) << 1) | (((v >> 6) >> 2) << 2);
    const bool leaf = !((A.mask[g] >> o) & 1u);
    const unsigned bal = __ballot_sync(0xffffffffu, leaf);
    if (lane == 0) wsum[w] = __popc(bal);
    __syncthreads();
    uint32_t before = 0;
    for (int k = 0; k < w; ++k) before += wsum[k];
    before += __popc(bal & ((1u << lane) - 1u));
    const uint32_t id = A.base[g] + before;
    A.leaf_of[g * TGV_BVOX + v] = leaf ? (int32_t)id : -1;
    if (leaf) {
        const int l = cb_level_of_brick(A, g);
        A.slot[id] = (int32_t)((g - A.L[l].bfirst) * TGV_BVOX + v);
    }
}

// forward (kind 0) and backward (kind 1) lists of every leaf
__global__ void cb_lists_kernel(const CBArgs A)
{
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < A.n; x += (int64_t)gridDim.x * blockDim.x) {
        const int l = cb_level_of_leaf(A, x);
        const CBLevel& L = A.L[l];
        const int64_t s = A.slot[x], b = s / TGV_BVOX, v = s % TGV_BVOX;
        const int64_t gv[3] = {8 * (int64_t)L.coords[3 * b] + (v & 7), 8 * (int64_t)L.coords[3 * b + 1] + ((v >> 3) & 7),
                               8 * (int64_t)L.coords[3 * b + 2] + (v >> 6)};
        for (int a = 0; a < 3; ++a)
            for (int side = 0; side < 2; ++side) {
                int64_t qv[3] = {gv[0], gv[1], gv[2]};
                qv[a] += side == 0 ? 1 : -1;
                int32_t* dst = A.lists + ((x * 4 + side) * 3 + a) * kList;
                const int64_t same = cb_leaf(A, l, qv[0], qv[1], qv[2]);
                if (same >= 0) {
                    dst[0] = (int32_t)same;
                } else if (same == -1) {  // refined: the 4 children on the face next to x
                    int64_t c0[3] = {2 * qv[0], 2 * qv[1], 2 * qv[2]};
                    if (side == 1) c0[a] += 1;
                    const int o0 = a == 0 ? 1 : 0, o1 = a == 2 ? 1 : 2;
                    int m = 0;
                    for (int d1 = 0; d1 < 2; ++d1)
                        for (int d0 = 0; d0 < 2; ++d0) {
                            int64_t cc[3] = {c0[0], c0[1], c0[2]};
                            cc[o0] += d0;
                            cc[o1] += d1;
                            const int64_t f = cb_leaf(A, l + 1, cc[0], cc[1], cc[2]);
                            if (f < 0) atomicAdd(&A.err[0], 1u);
                            else dst[m++] = (int32_t)f;
                        }
                } else if (l > 0) {
                    const int64_t cr = cb_leaf(A, l - 1, qv[0] >> 1, qv[1] >> 1, qv[2] >> 1);
                    if (cr >= 0) dst[0] = (int32_t)cr;
                }
            }
    }
}

// reverse lists: each leaf enters the +a (-a) reverse list of the leaves in its +a
// (-a) list, with weight 1 / (list length), into the first free of four slots
__global__ void cb_reverse_kernel(const CBArgs A)
{
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < A.n; x += (int64_t)gridDim.x * blockDim.x)
        for (int side = 0; side < 2; ++side)
            for (int a = 0; a < 3; ++a) {
                const int32_t* src = A.lists + ((x * 4 + side) * 3 + a) * kList;
                int cnt = 0;
                while (cnt < kList && src[cnt] >= 0) ++cnt;
                for (int k = 0; k < cnt; ++k) {
                    int* rev = (int*)(A.lists + (((int64_t)src[k] * 4 + 2 + side) * 3 + a) * kList);
                    const int val = (int)((uint32_t)x | (cnt == 4 ? kQuarter : 0u));
                    int m = 0;
                    while (m < kList && atomicCAS(rev + m, -1, val) != -1) ++m;
                    if (m == kList) atomicAdd(&A.err[1], 1u);
                }
            }
}

// reverse lists in leaf order; regular leaves get their six ids, irregular ones a mark
__global__ void cb_classify_kernel(const CBArgs A, uint32_t* irr)
{
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < A.n; x += (int64_t)gridDim.x * blockDim.x) {
        int32_t* L0 = A.lists + x * 4 * 3 * kList;
        for (int r = 6; r < 12; ++r) {  // kinds 2, 3: insertion sort by leaf id
            int32_t* e = L0 + r * kList;
            for (int i = 1; i < kList && e[i] != -1; ++i) {
                const int32_t key = e[i];
                int j = i - 1;
                while (j >= 0 && (e[j] & 0x7fffffff) > (key & 0x7fffffff)) {
                    e[j + 1] = e[j];
                    --j;
                }
                e[j + 1] = key;
            }
        }
        bool regular = true;
        for (int a = 0; a < 3 && regular; ++a) {
            const int32_t* f = L0 + (0 * 3 + a) * kList;
            const int32_t* bk = L0 + (1 * 3 + a) * kList;
            const int32_t* rf = L0 + (2 * 3 + a) * kList;
            const int32_t* rb = L0 + (3 * 3 + a) * kList;
            regular = f[1] < 0 && bk[1] < 0 && rf[1] == -1 && rb[1] == -1 && rf[0] == bk[0] && rb[0] == f[0];
        }
        if (regular) {
            for (int a = 0; a < 3; ++a) {
                A.nb6[x * 6 + a] = L0[(0 * 3 + a) * kList];
                A.nb6[x * 6 + 3 + a] = L0[(1 * 3 + a) * kList];
            }
        }
        irr[x] = regular ? 0u : 1u;
    }
}

// irregular leaves: their index among the irregular ones (scanned flags) and full lists
__global__ void cb_irregular_kernel(const CBArgs A, const uint32_t* irr_idx, int32_t* irr_lists, int64_t nirr)
{
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < A.n; x += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = irr_idx[x];
        const bool is_irr = x + 1 < A.n ? irr_idx[x + 1] > k : (int64_t)k < nirr;
        if (!is_irr) continue;
        A.nb6[x * 6] = (int32_t)(-2 - (int64_t)k);
        const int32_t* L0 = A.lists + x * 4 * 3 * kList;
        for (int i = 0; i < 4 * 3 * kList; ++i) irr_lists[(int64_t)k * 4 * 3 * kList + i] = L0[i];
    }
}

unsigned grid_of(int64_t n, int sms) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)sms * 32)); }

void free_comp(tgv_composite* c)
{
    for (void* p : {(void*)c->u, (void*)c->ubar, (void*)c->v, (void*)c->vbar, (void*)c->p, (void*)c->q, (void*)c->hist,
                    (void*)c->lists, (void*)c->nb6, (void*)c->slot, (void*)c->tt_part})
        if (p) cudaFree(p);
}

// ---- treetop (Sec. 4.3): the leaves in Z-order, split into the subtrees of the
// shallowest nodes that hold fewer than N of them

struct TTKeyArgs {
    const int32_t* slot;
    const int32_t* coords[32];
    int64_t lfirst[33];
    int nlev, root_bits, ib;
    int64_t n;
    uint64_t* keys;
    unsigned int* err;
};

// key of leaf i: Morton code of its lower corner in finest-level voxel units, above
// the leaf index (ib bits)
__global__ void tt_key_kernel(const TTKeyArgs A)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += (int64_t)gridDim.x * blockDim.x) {
        int l = 0;
        while (l + 1 < A.nlev && i >= A.lfirst[l + 1]) ++l;
        const int32_t sl = A.slot[i];
        const int32_t* cb = A.coords[l] + 3 * (int64_t)(sl >> 9);
        const int loc = sl & 511, sh = A.nlev - 1 - l;
        const int64_t g[3] = {8 * (int64_t)cb[0] + (loc & 7), 8 * (int64_t)cb[1] + ((loc >> 3) & 7),
                              8 * (int64_t)cb[2] + (loc >> 6)};
        bool ok = true;
        for (int a = 0; a < 3; ++a) ok = ok && g[a] >= 0 && ((g[a] << sh) >> A.root_bits) == 0;
        if (!ok) {
            atomicOr(A.err, 1u);
            A.keys[i] = 0;
            continue;
        }
        A.keys[i] = (morton3((uint64_t)g[0] << sh, (uint64_t)g[1] << sh, (uint64_t)g[2] << sh) << A.ib) | (uint64_t)i;
    }
}

// first position in [lo, hi) of the sorted keys at or after child c of node k
// (children at depth d + 1: code (node << 3) | c, `shift` = 3 (root_bits - d - 1) + ib)
__global__ void tt_split_kernel(const uint64_t* keys, int shift, const uint64_t* code, const int64_t* lo,
                                const int64_t* hi, int64_t nnodes, int64_t* lb)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 8 * nnodes) return;
    const int64_t k = t >> 3;
    const uint64_t target = (code[k] << 3) | (uint64_t)(t & 7);
    int64_t a = lo[k], b = hi[k];
    while (a < b) {
        const int64_t m = a + ((b - a) >> 1);
        if ((keys[m] >> shift) < target) a = m + 1;
        else b = m;
    }
    lb[t] = a;
}

// part[leaf] = the part whose Z-range holds the leaf's position
__global__ void tt_part_kernel(const uint64_t* keys, int64_t n, uint64_t idx_mask, const int64_t* first, int64_t nparts,
                               int32_t* part)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t a = 0, b = nparts;  // first index with first[.] > i, minus one
        while (a < b) {
            const int64_t m = a + ((b - a) >> 1);
            if (first[m] <= i) a = m + 1;
            else b = m;
        }
        part[keys[i] & idx_mask] = (int32_t)(a - 1);
    }
}

}  // namespace

extern "C" {

tgv_status tgv_composite_create(tgv_domain* d, tgv_composite** out)
{
    if (!out) return TGV_ERR_INVALID_ARG;
    *out = nullptr;
    if (!d) return TGV_ERR_INVALID_ARG;
    if (d->broken) return TGV_ERR_STATE;
    const int nlev = (int)d->levels.size();
    if (nlev > 32) return TGV_ERR_UNSUPPORTED;
    std::unique_ptr<tgv_composite> c(new (std::nothrow) tgv_composite());
    if (!c) return TGV_ERR_OUT_OF_MEMORY;
    c->d = d;
    cudaStream_t st = d->stream;
    CBArgs A;
    A.nlev = nlev;
    int64_t nbt = 0;
    uint64_t hcap_total = 0;
    for (int l = 0; l < nlev; ++l) {
        const TgvLevel& L = d->levels[l];
        A.L[l].coords = L.coords_dev;
        A.L[l].nb = L.nb;
        A.L[l].bfirst = nbt;
        uint64_t cap = 16;
        while (cap < 2 * (uint64_t)L.nb) cap <<= 1;
        A.L[l].hoff = hcap_total;
        A.L[l].hcap = cap;
        A.L[l].lfirst = 0;
        hcap_total += cap;
        nbt += L.nb;
    }
    if (nbt * TGV_BVOX >= ((int64_t)1 << 31) - 1) return TGV_ERR_UNSUPPORTED;
    A.nbt = nbt;
    // temporaries of the build
    struct Tmp {
        void* p = nullptr;
        ~Tmp()
        {
            if (p) cudaFree(p);
        }
    } hkeys, hvals, base, mask, leaf_of, lists, err, irr;
    auto alloc = [&](void** p, size_t bytes) {
        if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
            cudaGetLastError();
            *p = nullptr;
            return false;
        }
        return true;
    };
    const size_t nbz = (size_t)std::max<int64_t>(nbt, 1);
    if (!alloc(&hkeys.p, hcap_total * 8) || !alloc(&hvals.p, hcap_total * 4) || !alloc(&base.p, nbz * 4) ||
        !alloc(&mask.p, nbz) || !alloc(&leaf_of.p, nbz * TGV_BVOX * 4) || !alloc(&err.p, 16))
        return tgv_fail(d, TGV_ERR_OUT_OF_MEMORY, "composite build allocation failed");
    A.hkeys = (uint64_t*)hkeys.p;
    A.hvals = (int32_t*)hvals.p;
    A.base = (uint32_t*)base.p;
    A.mask = (uint8_t*)mask.p;
    A.leaf_of = (int32_t*)leaf_of.p;
    A.err = (unsigned int*)err.p;
    A.slot = nullptr;
    A.lists = nullptr;
    A.nb6 = nullptr;
    A.n = 0;
    cudaError_t e = cudaMemsetAsync(hkeys.p, 0xff, hcap_total * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(err.p, 0, 16, st);
    const unsigned bgrid = grid_of(nbt, d->sm_count);
    if (e == cudaSuccess && nbt > 0) {
        cb_insert_kernel<<<bgrid, 256, 0, st>>>(A);
        cb_mask_kernel<<<bgrid, 256, 0, st>>>(A);
        c->launches += 2;
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return tgv_cuda_check(d, e, "composite brick tables");
    // leaf numbering: exclusive scan of the leaf counts over all bricks
    uint64_t n = 0;
    TgvScratch scan_tmp;
    tgv_status s0 = nbt > 0 ? tgv_exclusive_scan_u32(d, A.base, nbt, scan_tmp, &n) : TGV_OK;
    std::vector<uint32_t> base_h((size_t)nbt);
    if (s0 == TGV_OK && nbt > 0) {
        e = cudaMemcpyAsync(base_h.data(), A.base, (size_t)nbt * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s0 = tgv_cuda_check(d, e, "composite leaf numbering");
    }
    auto free_scan_tmp = [&]() {
        if (scan_tmp.ptr) {
            cudaFree(scan_tmp.ptr);
            d->bytes -= (int64_t)scan_tmp.cap;
        }
        scan_tmp.ptr = nullptr;
        scan_tmp.cap = 0;
    };
    free_scan_tmp();
    if (s0 != TGV_OK) return s0;
    unsigned int herr[4] = {0, 0, 0, 0};
    for (int l = 0; l < nlev; ++l) {
        A.L[l].lfirst = A.L[l].bfirst < nbt ? (int64_t)base_h[(size_t)A.L[l].bfirst] : (int64_t)n;
        c->level_first.push_back(A.L[l].lfirst);
    }
    c->level_first.push_back((int64_t)n);
    c->n = (int64_t)n;
    A.n = (int64_t)n;
    const size_t nn = (size_t)std::max<uint64_t>(n, 1);
    const int npairs = (d->prm.nbins + 1) / 2;
    if (!alloc((void**)&c->slot, nn * 4) || !alloc(&lists.p, nn * 4 * 3 * kList * 4) ||
        !alloc((void**)&c->nb6, nn * 6 * 4) || !alloc(&irr.p, nn * 4)) {
        free_comp(c.get());
        return tgv_fail(d, TGV_ERR_OUT_OF_MEMORY, "composite list allocation failed");
    }
    A.slot = c->slot;
    A.lists = (int32_t*)lists.p;
    A.nb6 = c->nb6;
    e = cudaMemsetAsync(lists.p, 0xff, nn * 4 * 3 * kList * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->nb6, 0xff, nn * 6 * 4, st);
    const unsigned lgrid = grid_of((int64_t)n, d->sm_count);
    if (e == cudaSuccess && nbt > 0) {
        cb_leaves_kernel<<<(unsigned)nbt, TGV_BVOX, 0, st>>>(A);
        c->launches++;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && n > 0) {
        cb_lists_kernel<<<lgrid, 256, 0, st>>>(A);
        cb_reverse_kernel<<<lgrid, 256, 0, st>>>(A);
        cb_classify_kernel<<<lgrid, 256, 0, st>>>(A, (uint32_t*)irr.p);
        c->launches += 3;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(herr, err.p, sizeof(herr), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        free_comp(c.get());
        return tgv_cuda_check(d, e, "composite lists");
    }
    if (herr[2]) {
        free_comp(c.get());
        return tgv_fail(d, TGV_ERR_BUDGET, "composite brick table full");
    }
    if (herr[0]) {
        free_comp(c.get());
        return tgv_fail(d, TGV_ERR_INVALID_ARG, "levels are not 2:1 nested (a refined voxel lacks a child)");
    }
    if (herr[1]) {
        free_comp(c.get());
        return tgv_fail(d, TGV_ERR_INVALID_ARG, "a leaf has more than four neighbours over a face");
    }
    // irregular leaves: number them and keep their full lists
    uint64_t nirr = 0;
    s0 = n > 0 ? tgv_exclusive_scan_u32(d, (uint32_t*)irr.p, (int64_t)n, scan_tmp, &nirr) : TGV_OK;
    free_scan_tmp();
    if (s0 != TGV_OK) {
        free_comp(c.get());
        return s0;
    }
    c->nirr = (int64_t)nirr;
    if (!alloc((void**)&c->lists, (size_t)nirr * 4 * 3 * kList * 4 + 16)) {
        free_comp(c.get());
        return tgv_fail(d, TGV_ERR_OUT_OF_MEMORY, "composite allocation failed");
    }
    if (n > 0) {
        cb_irregular_kernel<<<lgrid, 256, 0, st>>>(A, (const uint32_t*)irr.p, c->lists, (int64_t)nirr);
        c->launches++;
        e = cudaGetLastError();
    }
    // state of the leaves
    if (e == cudaSuccess &&
        (!alloc((void**)&c->u, nn * 4) || !alloc((void**)&c->ubar, nn * 4) || !alloc((void**)&c->v, nn * 12) ||
         !alloc((void**)&c->vbar, nn * 12) || !alloc((void**)&c->p, nn * 12) || !alloc((void**)&c->q, nn * 24) ||
         !alloc((void**)&c->hist, nn * npairs * 4))) {
        free_comp(c.get());
        return tgv_fail(d, TGV_ERR_OUT_OF_MEMORY, "composite allocation failed");
    }
    for (void* p : {(void*)c->v, (void*)c->vbar, (void*)c->p, (void*)c->q}) {
        const size_t bytes = p == c->q ? nn * 24 : nn * 12;
        if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, bytes, st);
    }
    // u, ubar and histograms of the leaves from their levels
    for (int l = 0; l < nlev && e == cudaSuccess; ++l) {
        const int64_t o = c->level_first[l], nl = c->level_first[l + 1] - o;
        if (nl == 0) continue;
        comp_gather_u<<<grid_of(nl, d->sm_count), 256, 0, st>>>(c->u + o, c->ubar + o, d->levels[l].u, c->slot + o, nl);
        comp_gather_hist<<<grid_of(nl * npairs, d->sm_count), 256, 0, st>>>(c->hist + o * npairs, d->levels[l].hist,
                                                                             c->slot + o, nl, npairs);
        c->launches += 2;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the build's temporaries are freed on return
    if (e != cudaSuccess) {
        free_comp(c.get());
        return tgv_cuda_check(d, e, "composite initialisation");
    }
    *out = c.release();
    return TGV_OK;
}

tgv_status tgv_composite_solve(tgv_composite* c, int32_t iterations)
{
    TgvNvtxRange nvtx_range_("tgv_composite_solve");
    if (!c || iterations < 0) return TGV_ERR_INVALID_ARG;
    tgv_domain* d = c->d;
    if (d->broken) return TGV_ERR_STATE;
    if (c->n == 0 || iterations == 0) return TGV_OK;
    CompArgs A;
    A.u = c->u;
    A.ubar = c->ubar;
    A.v = c->v;
    A.vbar = c->vbar;
    A.p = c->p;
    A.q = c->q;
    A.hist = c->hist;
    A.lists = c->lists;
    A.nb6 = c->nb6;
    A.n = c->n;
    A.nbins = d->prm.nbins;
    A.npairs = (d->prm.nbins + 1) / 2;
    A.clamp_u = d->prm.clamp_u;
    A.alpha1 = d->prm.alpha1;
    A.alpha0 = d->prm.alpha0;
    A.tau = d->prm.tau;
    A.sigma = d->prm.sigma;
    A.taulam = d->prm.tau * d->prm.lambda;
    tgv_bin_centres(d->prm, A.c);
    const unsigned grid = (unsigned)((c->n + 511) / 512);  // two leaves per thread
    for (int it = 0; it < iterations; ++it) {
        comp_dual_kernel<<<grid, 256, 0, d->stream>>>(A);
        switch (A.nbins) {
        case 8: comp_primal_kernel<8><<<grid, 256, 0, d->stream>>>(A); break;
        case 10: comp_primal_kernel<10><<<grid, 256, 0, d->stream>>>(A); break;
        case 12: comp_primal_kernel<12><<<grid, 256, 0, d->stream>>>(A); break;
        default: comp_primal_kernel<0><<<grid, 256, 0, d->stream>>>(A); break;
        }
        c->launches += 2;
    }
    return tgv_cuda_check(d, cudaGetLastError(), "composite iteration launch");
}

int64_t tgv_composite_leaves(const tgv_composite* c) { return c ? c->n : 0; }

int64_t tgv_composite_level_leaves(const tgv_composite* c, int32_t level)
{
    if (!c || level < 0 || level + 1 >= (int32_t)c->level_first.size()) return -1;
    return c->level_first[level + 1] - c->level_first[level];
}

tgv_status tgv_composite_extract(tgv_composite* c, float* u_out, int64_t count)
{
    if (!c || (!u_out && count > 0) || count != c->n) return TGV_ERR_INVALID_ARG;
    tgv_domain* d = c->d;
    cudaError_t e = cudaSuccess;
    if (count > 0) e = cudaMemcpyAsync(u_out, c->u, (size_t)count * 4, cudaMemcpyDefault, d->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    return tgv_cuda_check(d, e, "composite extract");
}

tgv_status tgv_composite_scatter(tgv_composite* c)
{
    if (!c) return TGV_ERR_INVALID_ARG;
    tgv_domain* d = c->d;
    if (d->broken) return TGV_ERR_STATE;
    cudaError_t e = cudaSuccess;
    for (size_t l = 0; l + 1 < c->level_first.size() && e == cudaSuccess; ++l) {
        const int64_t o = c->level_first[l], nl = c->level_first[l + 1] - o;
        if (nl == 0) continue;
        comp_scatter_u<<<grid_of(nl, d->sm_count), 256, 0, d->stream>>>(d->levels[l].u, c->u + o, c->slot + o, nl);
        c->launches++;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    return tgv_cuda_check(d, e, "composite scatter");
}

int64_t tgv_composite_launch_count(const tgv_composite* c) { return c ? c->launches : 0; }

tgv_status tgv_composite_treetop(tgv_composite* c, int32_t root_bits, int64_t max_cubes, int64_t* nparts)
{
    if (nparts) *nparts = 0;
    if (!c || !nparts || root_bits < 1 || root_bits > 21 || max_cubes < 2) return TGV_ERR_INVALID_ARG;
    tgv_domain* d = c->d;
    if (d->broken) return TGV_ERR_STATE;
    const int nlev = (int)c->level_first.size() - 1;
    const int64_t n = c->n;
    int ib = 1;
    while (((int64_t)1 << ib) < n) ++ib;
    if (3 * root_bits + ib > 64) return tgv_fail(d, TGV_ERR_UNSUPPORTED, "treetop keys exceed 64 bits");
    c->tt_depth.clear();
    c->tt_code.clear();
    c->tt_first.clear();
    c->tt_last.clear();
    if (c->tt_part) cudaFree(c->tt_part);
    c->tt_part = nullptr;
    cudaStream_t st = d->stream;
    struct Buf {
        void* p = nullptr;
        ~Buf()
        {
            if (p) cudaFree(p);
        }
    } keys, tmp, hist, err, nodes, lbuf;
    auto alloc = [&](void** p, size_t bytes) {
        if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
            cudaGetLastError();
            *p = nullptr;
            return false;
        }
        return true;
    };
    const size_t nn = (size_t)std::max<int64_t>(n, 1);
    if (!alloc(&keys.p, nn * 8) || !alloc(&tmp.p, nn * 8) ||
        !alloc(&hist.p, (size_t)tgv_radix_hist_words(n) * 4) || !alloc(&err.p, 16))
        return tgv_fail(d, TGV_ERR_OUT_OF_MEMORY, "treetop allocation failed");
    if (n == 0) {
        if (!alloc((void**)&c->tt_part, 16)) return tgv_fail(d, TGV_ERR_OUT_OF_MEMORY, "treetop allocation failed");
        return TGV_OK;
    }
    TTKeyArgs K;
    K.slot = c->slot;
    for (int l = 0; l < nlev; ++l) {
        K.coords[l] = d->levels[l].coords_dev;
        K.lfirst[l] = c->level_first[l];
    }
    K.lfirst[nlev] = n;
    K.nlev = nlev;
    K.root_bits = root_bits;
    K.ib = ib;
    K.n = n;
    K.keys = (uint64_t*)keys.p;
    K.err = (unsigned int*)err.p;
    cudaError_t e = cudaMemsetAsync(err.p, 0, 16, st);
    if (e == cudaSuccess) {
        tt_key_kernel<<<grid_of(n, d->sm_count), 256, 0, st>>>(K);
        c->launches++;
        e = cudaGetLastError();
    }
    unsigned int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err.p, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return tgv_cuda_check(d, e, "treetop keys");
    if (herr) return tgv_fail(d, TGV_ERR_INVALID_ARG, "treetop: a leaf lies outside the root cube");
    // Z-order: the Morton digits only (the sort is stable and the keys come in index order)
    e = tgv_radix_sort_u64((uint64_t*)keys.p, (uint64_t*)tmp.p, (uint32_t*)hist.p, n, ib, 3 * root_bits, st,
                           &c->launches);
    if (e != cudaSuccess) return tgv_cuda_check(d, e, "treetop sort");
    auto emit = [&](int32_t depth, uint64_t code, int64_t lo, int64_t hi) {
        c->tt_depth.push_back(depth);
        c->tt_code.push_back(code);
        c->tt_first.push_back(lo);
        c->tt_last.push_back(hi - 1);
    };
    // top-down: the children of every node holding >= max_cubes leaves, by binary search
    std::vector<uint64_t> fcode{0};
    std::vector<int64_t> flo{0}, fhi{n};
    if (n < max_cubes) {
        emit(0, 0, 0, n);
        fcode.clear();
    }
    for (int depth = 0; !fcode.empty(); ++depth) {
        const int64_t nf = (int64_t)fcode.size();
        if (depth >= root_bits) return tgv_fail(d, TGV_ERR_STATE, "treetop: a finest-level node holds several leaves");
        if (nodes.p) cudaFree(nodes.p);
        if (lbuf.p) cudaFree(lbuf.p);
        nodes.p = lbuf.p = nullptr;
        if (!alloc(&nodes.p, (size_t)nf * 24) || !alloc(&lbuf.p, (size_t)nf * 64))
            return tgv_fail(d, TGV_ERR_OUT_OF_MEMORY, "treetop allocation failed");
        uint64_t* dcode = (uint64_t*)nodes.p;
        int64_t* dlo = (int64_t*)(dcode + nf);
        int64_t* dhi = dlo + nf;
        std::vector<int64_t> lb((size_t)(8 * nf));
        e = cudaMemcpyAsync(dcode, fcode.data(), (size_t)nf * 8, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dlo, flo.data(), (size_t)nf * 8, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dhi, fhi.data(), (size_t)nf * 8, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) {
            tt_split_kernel<<<(unsigned)((8 * nf + 255) / 256), 256, 0, st>>>(
                (const uint64_t*)keys.p, 3 * (root_bits - depth - 1) + ib, dcode, dlo, dhi, nf, (int64_t*)lbuf.p);
            c->launches++;
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(lb.data(), lbuf.p, (size_t)nf * 64, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return tgv_cuda_check(d, e, "treetop split");
        std::vector<uint64_t> ncode;
        std::vector<int64_t> nlo, nhi;
        for (int64_t k = 0; k < nf; ++k)
            for (int ch = 0; ch < 8; ++ch) {
                const int64_t a = lb[(size_t)(8 * k + ch)], b = ch < 7 ? lb[(size_t)(8 * k + ch + 1)] : fhi[(size_t)k];
                if (b <= a) continue;
                const uint64_t cc = (fcode[(size_t)k] << 3) | (uint64_t)ch;
                if (b - a < max_cubes) {
                    emit(depth + 1, cc, a, b);
                } else {
                    ncode.push_back(cc);
                    nlo.push_back(a);
                    nhi.push_back(b);
                }
            }
        fcode.swap(ncode);
        flo.swap(nlo);
        fhi.swap(nhi);
    }
    // parts in Z-order (their ranges are disjoint), then each leaf's part
    const size_t np = c->tt_first.size();
    std::vector<size_t> ord(np);
    for (size_t k = 0; k < np; ++k) ord[k] = k;
    std::sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return c->tt_first[a] < c->tt_first[b]; });
    auto permute = [&](auto& v) {
        auto w = v;
        for (size_t k = 0; k < np; ++k) w[k] = v[ord[k]];
        v.swap(w);
    };
    permute(c->tt_depth);
    permute(c->tt_code);
    permute(c->tt_first);
    permute(c->tt_last);
    if (nodes.p) cudaFree(nodes.p);
    nodes.p = nullptr;
    if (!alloc(&nodes.p, np * 8) || !alloc((void**)&c->tt_part, nn * 4))
        return tgv_fail(d, TGV_ERR_OUT_OF_MEMORY, "treetop allocation failed");
    e = cudaMemcpyAsync(nodes.p, c->tt_first.data(), np * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        tt_part_kernel<<<grid_of(n, d->sm_count), 256, 0, st>>>((const uint64_t*)keys.p, n,
                                                                 ((uint64_t)1 << ib) - 1, (const int64_t*)nodes.p,
                                                                 (int64_t)np, c->tt_part);
        c->launches++;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return tgv_cuda_check(d, e, "treetop parts");
    *nparts = (int64_t)np;
    return TGV_OK;
}

tgv_status tgv_composite_treetop_parts(tgv_composite* c, int32_t* depth, uint64_t* code, int64_t* first,
                                       int64_t* last, int32_t* leaf_part)
{
    if (!c) return TGV_ERR_INVALID_ARG;
    if (!c->tt_part) return TGV_ERR_STATE;
    if (depth) std::copy(c->tt_depth.begin(), c->tt_depth.end(), depth);
    if (code) std::copy(c->tt_code.begin(), c->tt_code.end(), code);
    if (first) std::copy(c->tt_first.begin(), c->tt_first.end(), first);
    if (last) std::copy(c->tt_last.begin(), c->tt_last.end(), last);
    if (!leaf_part || c->n == 0) return TGV_OK;
    tgv_domain* d = c->d;
    cudaError_t e = cudaMemcpyAsync(leaf_part, c->tt_part, (size_t)c->n * 4, cudaMemcpyDefault, d->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    return tgv_cuda_check(d, e, "treetop parts copy");
}

void tgv_composite_destroy(tgv_composite* c)
{
    if (!c) return;
    cudaStreamSynchronize(c->d->stream);
    free_comp(c);
    delete c;
}

}  // extern "C"
