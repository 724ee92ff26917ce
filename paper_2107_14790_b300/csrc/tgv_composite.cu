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
#include <math.h>

#include <memory>
#include <unordered_map>
#include <vector>

#include "tgv_internal.cuh"

struct tgv_composite {
    tgv_domain* d = nullptr;
    int64_t n = 0;
    std::vector<int64_t> level_first;             // first leaf of each level (and the total)
    std::vector<std::vector<int32_t>> leaf_slot;  // per level: slot (brick * 512 + local) of each leaf
    float *u = nullptr, *ubar = nullptr, *v = nullptr, *vbar = nullptr, *p = nullptr, *q = nullptr;
    uint32_t* hist = nullptr;                     // [n][npairs]
    int32_t* nb6 = nullptr;                       // [n][6]: +x +y +z -x -y -z neighbour of a regular leaf
    int32_t* lists = nullptr;                     // [irregular][4 kinds][3 axes][4]: fwd, bwd, rev fwd, rev bwd
    int64_t nirr = 0;
    int64_t launches = 0;
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
__global__ void comp_dual_kernel(const CompArgs A)
{
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
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

__device__ __forceinline__ int qidx_c(int a, int b) { return a == b ? a : (a + b == 1 ? 3 : (a + b == 2 ? 4 : 5)); }

__global__ void comp_primal_kernel(const CompArgs A)
{
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
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
    float hs = 0.0f, hb_[TGV_MAX_BINS];
    for (int k = 0; k < TGV_MAX_BINS; ++k) {
        hb_[k] = 0.0f;
        if (k < A.nbins) {
            const uint32_t w = A.hist[x * A.npairs + (k >> 1)];
            hb_[k] = (float)((w >> ((k & 1) * 16)) & 0xffffu);
            hs += hb_[k];
        }
    }
    float W = -hs, un = -INFINITY;
    for (int i = 0; i < TGV_MAX_BINS; ++i) {
        if (i < A.nbins) {
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

inline uint64_t ckey(int64_t x, int64_t y, int64_t z)
{
    const int64_t B = (int64_t)1 << 20;
    return ((uint64_t)(z + B) * (uint64_t)(2 * B) + (uint64_t)(y + B)) * (uint64_t)(2 * B) + (uint64_t)(x + B);
}

inline int64_t fdiv(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

unsigned grid_of(int64_t n, int sms) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)sms * 32)); }

void free_comp(tgv_composite* c)
{
    for (void* p : {(void*)c->u, (void*)c->ubar, (void*)c->v, (void*)c->vbar, (void*)c->p, (void*)c->q, (void*)c->hist,
                    (void*)c->lists, (void*)c->nb6})
        if (p) cudaFree(p);
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
    // brick index per level, and leaf ids
    std::vector<std::unordered_map<uint64_t, int64_t>> bidx(nlev);
    for (int l = 0; l < nlev; ++l) {
        const TgvLevel& L = d->levels[l];
        bidx[l].reserve((size_t)L.nb * 2);
        for (int64_t b = 0; b < L.nb; ++b) bidx[l].emplace(ckey(L.coords[3 * b], L.coords[3 * b + 1], L.coords[3 * b + 2]), b);
    }
    auto brick_at = [&](int l, int64_t x, int64_t y, int64_t z) -> int64_t {
        if (l < 0 || l >= nlev) return -1;
        auto it = bidx[l].find(ckey(fdiv(x, 8), fdiv(y, 8), fdiv(z, 8)));
        return it == bidx[l].end() ? -1 : it->second;
    };
    std::unique_ptr<tgv_composite> c(new (std::nothrow) tgv_composite());
    if (!c) return TGV_ERR_OUT_OF_MEMORY;
    c->d = d;
    c->leaf_slot.resize(nlev);
    std::vector<std::vector<int32_t>> leaf_id(nlev);  // per level slot -> leaf id (-1: refined)
    int64_t n = 0;
    for (int l = 0; l < nlev; ++l) {
        const TgvLevel& L = d->levels[l];
        c->level_first.push_back(n);
        leaf_id[l].assign((size_t)L.nb * TGV_BVOX, -1);
        for (int64_t b = 0; b < L.nb; ++b) {
            bool fine[8];
            for (int o = 0; o < 8; ++o)
                fine[o] = brick_at(l + 1, 16 * (int64_t)L.coords[3 * b] + 8 * (o & 1),
                                   16 * (int64_t)L.coords[3 * b + 1] + 8 * ((o >> 1) & 1),
                                   16 * (int64_t)L.coords[3 * b + 2] + 8 * (o >> 2)) >= 0;
            for (int v = 0; v < TGV_BVOX; ++v) {
                const int o = ((v & 7) >> 2) | ((((v >> 3) & 7) >> 2) << 1) | (((v >> 6) >> 2) << 2);
                if (fine[o]) continue;
                leaf_id[l][(size_t)b * TGV_BVOX + v] = (int32_t)n++;
                c->leaf_slot[l].push_back((int32_t)(b * TGV_BVOX + v));
            }
        }
        if (n >= ((int64_t)1 << 31) - 1) return TGV_ERR_UNSUPPORTED;
    }
    c->level_first.push_back(n);
    c->n = n;
    // neighbour lists
    std::vector<int32_t> lists((size_t)n * 4 * 3 * kList, -1);
    auto leaf_of = [&](int l, int64_t x, int64_t y, int64_t z) -> int64_t {
        const int64_t b = brick_at(l, x, y, z);
        if (b < 0) return -2;  // no voxel at this level
        return leaf_id[l][(size_t)b * TGV_BVOX + (x - 8 * fdiv(x, 8)) + 8 * (y - 8 * fdiv(y, 8)) + 64 * (z - 8 * fdiv(z, 8))];
    };
    bool ok = true;
    for (int l = 0; l < nlev && ok; ++l) {
        const TgvLevel& L = d->levels[l];
        for (size_t k = 0; k < c->leaf_slot[l].size() && ok; ++k) {
            const int64_t s = c->leaf_slot[l][k], b = s / TGV_BVOX, v = s % TGV_BVOX;
            const int64_t g[3] = {8 * (int64_t)L.coords[3 * b] + (v & 7), 8 * (int64_t)L.coords[3 * b + 1] + ((v >> 3) & 7),
                                  8 * (int64_t)L.coords[3 * b + 2] + (v >> 6)};
            const int64_t x = c->level_first[l] + (int64_t)k;
            for (int a = 0; a < 3; ++a)
                for (int side = 0; side < 2; ++side) {
                    int64_t qv[3] = {g[0], g[1], g[2]};
                    qv[a] += side == 0 ? 1 : -1;
                    int32_t* dst = &lists[(((size_t)x * 4 + side) * 3 + a) * kList];
                    const int64_t same = leaf_of(l, qv[0], qv[1], qv[2]);
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
                                const int64_t f = leaf_of(l + 1, cc[0], cc[1], cc[2]);
                                if (f < 0) ok = false;
                                else dst[m++] = (int32_t)f;
                            }
                    } else if (l > 0) {
                        const int64_t cr = leaf_of(l - 1, qv[0] >> 1, qv[1] >> 1, qv[2] >> 1);
                        if (cr >= 0) dst[0] = (int32_t)cr;
                    }
                }
        }
    }
    if (!ok) return tgv_fail(d, TGV_ERR_INVALID_ARG, "levels are not 2:1 nested (a refined voxel lacks a child)");
    // reverse lists: leaves whose +a (-a) list holds x, with weight 1 / list length
    for (int64_t x = 0; x < n && ok; ++x)
        for (int side = 0; side < 2; ++side)
            for (int a = 0; a < 3; ++a) {
                const int32_t* src = &lists[(((size_t)x * 4 + side) * 3 + a) * kList];
                int cnt = 0;
                while (cnt < kList && src[cnt] >= 0) ++cnt;
                for (int k = 0; k < cnt; ++k) {
                    int32_t* rev = &lists[(((size_t)src[k] * 4 + 2 + side) * 3 + a) * kList];
                    int m = 0;
                    while (m < kList && rev[m] != -1) ++m;
                    if (m == kList) {
                        ok = false;
                        break;
                    }
                    rev[m] = (int32_t)((uint32_t)x | (cnt == 4 ? kQuarter : 0u));
                }
            }
    if (!ok) return tgv_fail(d, TGV_ERR_INVALID_ARG, "a leaf has more than four neighbours over a face");
    // regular leaves: at most one neighbour per side and mirrored reverse lists of weight 1
    std::vector<int32_t> nb6((size_t)n * 6, -1), irr_lists;
    int64_t nirr = 0;
    for (int64_t x = 0; x < n; ++x) {
        const int32_t* L0 = &lists[(size_t)x * 4 * 3 * kList];
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
                nb6[(size_t)x * 6 + a] = L0[(0 * 3 + a) * kList];
                nb6[(size_t)x * 6 + 3 + a] = L0[(1 * 3 + a) * kList];
            }
        } else {
            nb6[(size_t)x * 6] = (int32_t)(-2 - nirr);
            irr_lists.insert(irr_lists.end(), L0, L0 + 4 * 3 * kList);
            ++nirr;
        }
    }
    c->nirr = nirr;
    std::vector<int32_t>().swap(lists);
    const int npairs = (d->prm.nbins + 1) / 2;
    cudaStream_t st = d->stream;
    auto alloc = [&](void** p, size_t bytes) {
        if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
            cudaGetLastError();
            *p = nullptr;
            return false;
        }
        return true;
    };
    const size_t nn = (size_t)std::max<int64_t>(n, 1);
    if (!alloc((void**)&c->u, nn * 4) || !alloc((void**)&c->ubar, nn * 4) || !alloc((void**)&c->v, nn * 12) ||
        !alloc((void**)&c->vbar, nn * 12) || !alloc((void**)&c->p, nn * 12) || !alloc((void**)&c->q, nn * 24) ||
        !alloc((void**)&c->hist, nn * npairs * 4) || !alloc((void**)&c->lists, irr_lists.size() * 4 + 16) ||
        !alloc((void**)&c->nb6, nb6.size() * 4)) {
        free_comp(c.get());
        return tgv_fail(d, TGV_ERR_OUT_OF_MEMORY, "composite allocation failed");
    }
    cudaError_t e = cudaMemcpyAsync(c->nb6, nb6.data(), nb6.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !irr_lists.empty())
        e = cudaMemcpyAsync(c->lists, irr_lists.data(), irr_lists.size() * 4, cudaMemcpyHostToDevice, st);
    for (void* p : {(void*)c->v, (void*)c->vbar, (void*)c->p, (void*)c->q}) {
        const size_t bytes = p == c->q ? nn * 24 : nn * 12;
        if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, bytes, st);
    }
    // u, ubar and histograms of the leaves from their levels
    int32_t* slots = nullptr;
    if (e == cudaSuccess && !alloc((void**)&slots, nn * 4)) e = cudaErrorMemoryAllocation;
    for (int l = 0; l < nlev && e == cudaSuccess; ++l) {
        const int64_t nl = (int64_t)c->leaf_slot[l].size();
        if (nl == 0) continue;
        e = cudaMemcpyAsync(slots, c->leaf_slot[l].data(), (size_t)nl * 4, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) break;
        const int64_t o = c->level_first[l];
        comp_gather_u<<<grid_of(nl, d->sm_count), 256, 0, st>>>(c->u + o, c->ubar + o, d->levels[l].u, slots, nl);
        comp_gather_hist<<<grid_of(nl * npairs, d->sm_count), 256, 0, st>>>(c->hist + o * npairs, d->levels[l].hist,
                                                                             slots, nl, npairs);
        c->launches += 2;
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // `slots` is reused for the next level
    }
    if (slots) cudaFree(slots);
    if (e != cudaSuccess) {
        free_comp(c.get());
        return tgv_cuda_check(d, e, "composite initialisation");
    }
    *out = c.release();
    return TGV_OK;
}

tgv_status tgv_composite_solve(tgv_composite* c, int32_t iterations)
{
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
    const unsigned grid = (unsigned)((c->n + 255) / 256);
    for (int it = 0; it < iterations; ++it) {
        comp_dual_kernel<<<grid, 256, 0, d->stream>>>(A);
        comp_primal_kernel<<<grid, 256, 0, d->stream>>>(A);
        c->launches += 2;
    }
    return tgv_cuda_check(d, cudaGetLastError(), "composite iteration launch");
}

int64_t tgv_composite_leaves(const tgv_composite* c) { return c ? c->n : 0; }

int64_t tgv_composite_level_leaves(const tgv_composite* c, int32_t level)
{
    if (!c || level < 0 || level >= (int32_t)c->leaf_slot.size()) return -1;
    return (int64_t)c->leaf_slot[level].size();
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
    int32_t* slots = nullptr;
    const size_t nn = (size_t)std::max<int64_t>(c->n, 1);
    if (cudaMalloc(&slots, nn * 4) != cudaSuccess) {
        cudaGetLastError();
        return tgv_fail(d, TGV_ERR_OUT_OF_MEMORY, "composite scatter scratch");
    }
    cudaError_t e = cudaSuccess;
    for (size_t l = 0; l < c->leaf_slot.size() && e == cudaSuccess; ++l) {
        const int64_t nl = (int64_t)c->leaf_slot[l].size();
        if (nl == 0) continue;
        e = cudaMemcpyAsync(slots, c->leaf_slot[l].data(), (size_t)nl * 4, cudaMemcpyHostToDevice, d->stream);
        if (e != cudaSuccess) break;
        comp_scatter_u<<<grid_of(nl, d->sm_count), 256, 0, d->stream>>>(d->levels[l].u, c->u + c->level_first[l],
                                                                        slots, nl);
        c->launches++;
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    }
    cudaFree(slots);
    return tgv_cuda_check(d, e, "composite scatter");
}

int64_t tgv_composite_launch_count(const tgv_composite* c) { return c ? c->launches : 0; }

void tgv_composite_destroy(tgv_composite* c)
{
    if (!c) return;
    cudaStreamSynchronize(c->d->stream);
    free_comp(c);
    delete c;
}

}  // extern "C"
