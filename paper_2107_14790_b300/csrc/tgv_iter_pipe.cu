// Pipelined form of the fused TGV primal-dual iteration (the arithmetic of
// tgv_iter_kernel in tgv_solve.cu: Eq. 2-3, Sec. 3.2).
//
// Persistent CTAs (512 threads, one per voxel of the brick in hand) walk the
// active bricks with a grid stride.  Each brick's whole state -- u, ubar, v,
// vbar, p, q and the packed histogram, all contiguous per brick -- arrives in
// shared memory through seven cp.async.bulk copies completed on an mbarrier,
// double-buffered: while brick i is computed, brick i + grid is in flight.
// Halo values owned by neighbouring bricks (one face layer of ubar / vbar / p / q
// and one edge line of ubar / vbar) are loaded into registers before the CTA
// waits for its stage, so their latency overlaps the stage's.
//
// The bin count is a template parameter for the common 8, 10 and 12 bins
// (0 = read at run time).
//
// Every mbarrier wait is bounded (about a second); a CTA that gives up sets
// the domain's error flag, waits (bounded) for its copies still in flight and
// returns.
#include <math.h>

#include "tgv_async.cuh"
#include "tgv_internal.cuh"

namespace {

__device__ __forceinline__ int qidx(int a, int b) { return a == b ? a : (a + b == 1 ? 3 : (a + b == 2 ? 4 : 5)); }

__device__ __forceinline__ int face_idx(int a, int x, int y, int z)
{
    return a == 0 ? y + 8 * z : (a == 1 ? x + 8 * z : x + 8 * y);
}

__host__ __device__ constexpr int kStride(int a) { return a == 0 ? 1 : (a == 1 ? 8 : 64); }

// The two face axes of axis A, lower first.
template <int A> struct FaceAxes {
    static constexpr int B1 = A == 0 ? 1 : 0;
    static constexpr int B2 = A == 2 ? 1 : 2;
};

// ---- halo p on the -A face: voxel (coordinate 7 along A in brick n); loads before the stage wait
template <typename S, typename D, int A>
__device__ __forceinline__ void halo_p_load(const IterArgs<S, D>& P, const int* nrow, uint32_t n, int k, float hr[15],
                                            uint32_t& hmask)
{
    constexpr int B1 = FaceAxes<A>::B1, B2 = FaceAxes<A>::B2;
    const int c1 = k & 7, c2 = k >> 3;
    const uint32_t lh = 7 * kStride(A) + c1 * kStride(B1) + c2 * kStride(B2);
    const size_t nb0 = (size_t)n * TGV_BVOX;
    hr[0] = P.ubar_in[nb0 + lh];
    if (c1 < 7) {
        hr[1] = P.ubar_in[nb0 + lh + kStride(B1)];
        hmask |= 1u;
    } else {
        const int e = nrow[nb_edge(A, B1)];
        if (e >= 0) {
            hr[1] = P.ubar_in[(size_t)e * TGV_BVOX + lh - 7 * kStride(B1)];
            hmask |= 1u;
        }
    }
    if (c2 < 7) {
        hr[2] = P.ubar_in[nb0 + lh + kStride(B2)];
        hmask |= 2u;
    } else {
        const int e = nrow[nb_edge(A, B2)];
        if (e >= 0) {
            hr[2] = P.ubar_in[(size_t)e * TGV_BVOX + lh - 7 * kStride(B2)];
            hmask |= 2u;
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        hr[3 + c] = ld_s(P.vbar_in + ((size_t)n * 3 + c) * TGV_BVOX + lh);
        hr[6 + c] = ld_d(P.p_in + ((size_t)n * 3 + c) * TGV_BVOX + lh, P.ds.dsp);
    }
}

template <typename S, typename D, int A>
__device__ __forceinline__ void halo_p_compute(const IterArgs<S, D>& P, const float* sub, float* hal_p, int k,
                                               const float hr[15], uint32_t hmask, float a1sq)
{
    constexpr int B1 = FaceAxes<A>::B1, B2 = FaceAxes<A>::B2;
    const int c1 = k & 7, c2 = k >> 3;
    const int lo = c1 * kStride(B1) + c2 * kStride(B2);  // own voxel at coordinate 0 along A
    float g[3];
    g[A] = sub[lo] - hr[0];
    g[B1] = (hmask & 1u) ? hr[1] - hr[0] : 0.0f;
    g[B2] = (hmask & 2u) ? hr[2] - hr[0] : 0.0f;
    float ph[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) ph[c] = hr[6 + c] + P.sigma * (g[c] - hr[3 + c]);
    const float n2 = ph[0] * ph[0] + ph[1] * ph[1] + ph[2] * ph[2];
    if (n2 > a1sq) {
        const float s = P.alpha1 * rsqrtf(n2);
        ph[0] *= s;
        ph[1] *= s;
        ph[2] *= s;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) hal_p[c * 192 + A * 64 + k] = ph[c];
}

// ---- halo q on the +A face: voxel (coordinate 0 along A in brick n)
template <typename S, typename D, int A>
__device__ __forceinline__ void halo_q_load(const IterArgs<S, D>& P, const int* nrow, uint32_t n, int k, float hr[15],
                                            uint32_t& hmask)
{
    constexpr int B1 = FaceAxes<A>::B1, B2 = FaceAxes<A>::B2;
    const int c1 = k & 7, c2 = k >> 3;
    const uint32_t lh = c1 * kStride(B1) + c2 * kStride(B2);
#pragma unroll
    for (int c = 0; c < 3; ++c) hr[c] = ld_s(P.vbar_in + ((size_t)n * 3 + c) * TGV_BVOX + lh);
    if (c1 > 0) {
#pragma unroll
        for (int c = 0; c < 3; ++c) hr[3 + c] = ld_s(P.vbar_in + ((size_t)n * 3 + c) * TGV_BVOX + lh - kStride(B1));
        hmask |= 1u;
    } else {
        const int e = nrow[nb_edge(B1, A)];  // offset +1 along A, -1 along B1
        if (e >= 0) {
#pragma unroll
            for (int c = 0; c < 3; ++c)
                hr[3 + c] = ld_s(P.vbar_in + ((size_t)e * 3 + c) * TGV_BVOX + lh + 7 * kStride(B1));
            hmask |= 1u;
        }
    }
    if (c2 > 0) {
#pragma unroll
        for (int c = 0; c < 3; ++c) hr[6 + c] = ld_s(P.vbar_in + ((size_t)n * 3 + c) * TGV_BVOX + lh - kStride(B2));
        hmask |= 2u;
    } else {
        const int e = nrow[nb_edge(B2, A)];
        if (e >= 0) {
#pragma unroll
            for (int c = 0; c < 3; ++c)
                hr[6 + c] = ld_s(P.vbar_in + ((size_t)e * 3 + c) * TGV_BVOX + lh + 7 * kStride(B2));
            hmask |= 2u;
        }
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) hr[9 + c] = ld_d(P.q_in + ((size_t)n * 6 + c) * TGV_BVOX + lh, P.ds.dsq);
}

template <typename S, typename D, int A>
__device__ __forceinline__ void halo_q_compute(const IterArgs<S, D>& P, const S* svb, float* hal_q, int k,
                                               const float hr[15], uint32_t hmask, float a0sq)
{
    constexpr int B1 = FaceAxes<A>::B1, B2 = FaceAxes<A>::B2;
    const int c1 = k & 7, c2 = k >> 3;
    const int lo = 7 * kStride(A) + c1 * kStride(B1) + c2 * kStride(B2);  // own voxel at coordinate 7 along A
    float dm[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        dm[A][c] = hr[c] - ld_s(svb + c * 512 + lo);
        dm[B1][c] = (hmask & 1u) ? hr[c] - hr[3 + c] : 0.0f;
        dm[B2][c] = (hmask & 2u) ? hr[c] - hr[6 + c] : 0.0f;
    }
    float qh[6] = {dm[0][0], dm[1][1], dm[2][2], 0.5f * (dm[0][1] + dm[1][0]), 0.5f * (dm[0][2] + dm[2][0]),
                   0.5f * (dm[1][2] + dm[2][1])};
#pragma unroll
    for (int c = 0; c < 6; ++c) qh[c] = hr[9 + c] + P.sigma * qh[c];
    const float n2 = qh[0] * qh[0] + qh[1] * qh[1] + qh[2] * qh[2] + 2.0f * (qh[3] * qh[3] + qh[4] * qh[4] + qh[5] * qh[5]);
    if (n2 > a0sq) {
        const float s = P.alpha0 * rsqrtf(n2);
#pragma unroll
        for (int c = 0; c < 6; ++c) qh[c] *= s;
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) hal_q[c * 192 + A * 64 + k] = qh[c];
}

}  // namespace

template <typename S, typename D>
struct PipeArgs {
    IterArgs<S, D> it;
    int* err;              // set to 1 when a bounded wait gives up
    long long wait_budget; // clock cycles per wait
    uint32_t stage_bytes;  // bytes of one stage (multiple of 128)
    uint32_t tx_bytes;     // bytes the seven copies of one stage deliver
    uint32_t off_pn, off_qn;      // own new p / q (float); unused when S is float (they alias the stage)
    uint32_t off_hp, off_hq;      // halo new p [3][192], q [6][192] (float)
    uint32_t off_nbr, off_bar;    // neighbour rows [2][12], mbarriers [2]
};

template <typename S, typename D, int NB>
__global__ void __launch_bounds__(512, 2) tgv_iter_pipe_kernel(const PipeArgs<S, D> P)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const IterArgs<S, D>& A = P.it;
    constexpr uint32_t SB = sizeof(S), SD = sizeof(D);
    constexpr uint32_t O_U = 0, O_UB = 2048, O_V = 4096, O_VB = O_V + 3 * 512 * SB, O_P = O_VB + 3 * 512 * SB,
                       O_Q = O_P + 3 * 512 * SD, O_H = O_Q + 6 * 512 * SD;
    constexpr int NP_MAX = NB ? (NB + 1) / 2 : TGV_MAX_BINS / 2;
    constexpr int NB_MAX = NB ? NB : TGV_MAX_BINS;
    const int nbins = NB ? NB : A.nbins;
    const int npairs = NB ? (NB + 1) / 2 : A.npairs;
    const int t = threadIdx.x;
    const int x = t & 7, y = (t >> 3) & 7, z = t >> 6;
    const int crd[3] = {x, y, z};
    const uint32_t G = gridDim.x;
    const uint32_t nbk = (uint32_t)A.nb;
    const uint32_t nit = (uint32_t)A.nitems;
    const int32_t* work = A.work;
    auto brick = [&](uint32_t i) -> uint32_t { return work ? (uint32_t)work[i] : i; };
    uint32_t it = blockIdx.x;
    uint64_t* bar = (uint64_t*)(smem + P.off_bar);
    int* s_nbr = (int*)(smem + P.off_nbr);
    float* hal_p = (float*)(smem + P.off_hp);
    float* hal_q = (float*)(smem + P.off_hq);
    const float a1sq = A.alpha1 * A.alpha1, a0sq = A.alpha0 * A.alpha0;

    auto issue = [&](int s, uint32_t brick) {
        unsigned char* st = smem + (size_t)s * P.stage_bytes;
        mbar_arrive_expect_tx(&bar[s], P.tx_bytes);
        bulk_copy_g2s(st + O_U, A.u + (size_t)brick * TGV_BVOX, 2048, &bar[s]);
        bulk_copy_g2s(st + O_UB, A.ubar_in + (size_t)brick * TGV_BVOX, 2048, &bar[s]);
        bulk_copy_g2s(st + O_V, A.v + (size_t)brick * 3 * TGV_BVOX, 3 * 512 * SB, &bar[s]);
        bulk_copy_g2s(st + O_VB, A.vbar_in + (size_t)brick * 3 * TGV_BVOX, 3 * 512 * SB, &bar[s]);
        bulk_copy_g2s(st + O_P, A.p_in + (size_t)brick * 3 * TGV_BVOX, 3 * 512 * SD, &bar[s]);
        bulk_copy_g2s(st + O_Q, A.q_in + (size_t)brick * 6 * TGV_BVOX, 6 * 512 * SD, &bar[s]);
        bulk_copy_g2s(st + O_H, A.hist + brick * (size_t)npairs * TGV_BVOX, (uint32_t)npairs * 2048u, &bar[s]);
    };

    if (t == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    if (t < TGV_NNBR) s_nbr[t] = A.nbr[brick(it) * TGV_NNBR + t];
    __syncthreads();
    if (t == 0) {
        issue(0, brick(it));
        if (it + G < nit) issue(1, brick(it + G));
    }

    uint32_t parity = 0;  // bit s: parity of the next phase of stage s
    int s = 0;
    bool bail = false;
    // halo task of this thread: t < 192 new p on the -a face, 192 <= t < 384 new q on the +a face
    const bool ptask = t < 192, qtask = t >= 192 && t < 384;
    const int ha = ptask ? (t >> 6) : ((t - 192) >> 6);
    const int hk = t & 63;
    for (; it < nit; it += G, s ^= 1) {
        const uint32_t b = brick(it);
        unsigned char* st = smem + (size_t)s * P.stage_bytes;
        const int* nrow = s_nbr + s * TGV_NNBR;

        // ---- loads that do not depend on the stage: own face neighbours and halo inputs
        uint32_t fmask = 0, bmask = 0;
        float ubf[3], vbb[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            ubf[a] = 0.0f;
            vbb[a][0] = vbb[a][1] = vbb[a][2] = 0.0f;
            if (crd[a] == 7) {
                const int n = nrow[nb_plus(a)];
                if (n >= 0) {
                    ubf[a] = A.ubar_in[(size_t)n * TGV_BVOX + t - 7 * kStride(a)];
                    fmask |= 1u << a;
                }
            } else {
                fmask |= 1u << a;
            }
            if (crd[a] == 0) {
                const int n = nrow[nb_minus(a)];
                if (n >= 0) {
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        vbb[a][c] = ld_s(A.vbar_in + ((size_t)n * 3 + c) * TGV_BVOX + t + 7 * kStride(a));
                    bmask |= 1u << a;
                }
            } else {
                bmask |= 1u << a;
            }
        }
        int hn = -1;
        if (ptask || qtask) {
            hn = nrow[ptask ? nb_minus(ha) : nb_plus(ha)];
            if (hn >= (int)nbk) hn = -1;  // frozen: no dual variables there
        }
        float hr[15];
        uint32_t hmask = 0;
#pragma unroll
        for (int k = 0; k < 15; ++k) hr[k] = 0.0f;
        if (hn >= 0) {
            if (ptask) {
                if (ha == 0) halo_p_load<S, D, 0>(A, nrow, (uint32_t)hn, hk, hr, hmask);
                else if (ha == 1) halo_p_load<S, D, 1>(A, nrow, (uint32_t)hn, hk, hr, hmask);
                else halo_p_load<S, D, 2>(A, nrow, (uint32_t)hn, hk, hr, hmask);
            } else {
                if (ha == 0) halo_q_load<S, D, 0>(A, nrow, (uint32_t)hn, hk, hr, hmask);
                else if (ha == 1) halo_q_load<S, D, 1>(A, nrow, (uint32_t)hn, hk, hr, hmask);
                else halo_q_load<S, D, 2>(A, nrow, (uint32_t)hn, hk, hr, hmask);
            }
        }
        // neighbour row of the next brick of this CTA (its previous user finished at the last barrier)
        if (t < TGV_NNBR && it + G < nit) s_nbr[(s ^ 1) * TGV_NNBR + t] = A.nbr[brick(it + G) * TGV_NNBR + t];

        // ---- wait for this brick's stage
        const bool ok = mbar_wait_bounded(&bar[s], (parity >> s) & 1u, P.wait_budget);
        if (__syncthreads_or(!ok)) {
            bail = true;
            break;
        }
        parity ^= 1u << s;

        const float* su = (const float*)(st + O_U);
        const float* sub = (const float*)(st + O_UB);
        const S* sv = (const S*)(st + O_V);
        const S* svb = (const S*)(st + O_VB);
        const D* sp = (const D*)(st + O_P);
        const D* sq = (const D*)(st + O_Q);
        const uint32_t* sh = (const uint32_t*)(st + O_H);
        float* pn_own = (float*)(SD == 4 ? st + O_P : smem + P.off_pn);
        float* qn_own = (float*)(SD == 4 ? st + O_Q : smem + P.off_qn);

        // ---- phase A: dual ascent + projection at the own voxel
        const float ub = sub[t];
        float vb[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) vb[c] = ld_s(svb + c * 512 + t);
        float pn[3], qn[6];
        {
            float g[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float nv = crd[a] < 7 ? sub[t + kStride(a)] : ubf[a];
                g[a] = (fmask >> a) & 1u ? nv - ub : 0.0f;
            }
            float dm[3][3];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float w = crd[a] > 0 ? ld_s(svb + c * 512 + t - kStride(a)) : vbb[a][c];
                    dm[a][c] = (bmask >> a) & 1u ? vb[c] - w : 0.0f;
                }
#pragma unroll
            for (int c = 0; c < 3; ++c) pn[c] = ld_d(sp + c * 512 + t, A.ds.dsp) + A.sigma * (g[c] - vb[c]);
            const float pn2 = pn[0] * pn[0] + pn[1] * pn[1] + pn[2] * pn[2];
            if (pn2 > a1sq) {
                const float sc = A.alpha1 * rsqrtf(pn2);
                pn[0] *= sc;
                pn[1] *= sc;
                pn[2] *= sc;
            }
            qn[0] = dm[0][0];
            qn[1] = dm[1][1];
            qn[2] = dm[2][2];
            qn[3] = 0.5f * (dm[0][1] + dm[1][0]);
            qn[4] = 0.5f * (dm[0][2] + dm[2][0]);
            qn[5] = 0.5f * (dm[1][2] + dm[2][1]);
#pragma unroll
            for (int c = 0; c < 6; ++c) qn[c] = ld_d(sq + c * 512 + t, A.ds.dsq) + A.sigma * qn[c];
            const float qn2 =
                qn[0] * qn[0] + qn[1] * qn[1] + qn[2] * qn[2] + 2.0f * (qn[3] * qn[3] + qn[4] * qn[4] + qn[5] * qn[5]);
            if (qn2 > a0sq) {
                const float sc = A.alpha0 * rsqrtf(qn2);
#pragma unroll
                for (int c = 0; c < 6; ++c) qn[c] *= sc;
            }
        }
        // the own old p / q were read above by this thread only; overwrite in place (FP32) or store
#pragma unroll
        for (int c = 0; c < 3; ++c) pn_own[c * 512 + t] = pn[c];
#pragma unroll
        for (int c = 0; c < 6; ++c) qn_own[c * 512 + t] = qn[c];

        // ---- halo duals
        if (hn >= 0) {
            if (ptask) {
                if (ha == 0) halo_p_compute<S, D, 0>(A, sub, hal_p, hk, hr, hmask, a1sq);
                else if (ha == 1) halo_p_compute<S, D, 1>(A, sub, hal_p, hk, hr, hmask, a1sq);
                else halo_p_compute<S, D, 2>(A, sub, hal_p, hk, hr, hmask, a1sq);
            } else {
                if (ha == 0) halo_q_compute<S, D, 0>(A, svb, hal_q, hk, hr, hmask, a0sq);
                else if (ha == 1) halo_q_compute<S, D, 1>(A, svb, hal_q, hk, hr, hmask, a0sq);
                else halo_q_compute<S, D, 2>(A, svb, hal_q, hk, hr, hmask, a0sq);
            }
        }
        __syncthreads();

        // ---- phase B: primal descent, prox, over-relaxation
        float div1 = 0.0f;
        float div2[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int np = crd[a] < 7 ? 0 : nrow[nb_plus(a)];
            const int nm = crd[a] > 0 ? 0 : nrow[nb_minus(a)];
            const bool fwd_any = np >= 0;
            const bool fwd_act = np >= 0 && (crd[a] < 7 || np < (int)nbk);
            const bool bwd_any = nm >= 0;
            const bool bwd_act = nm >= 0 && (crd[a] > 0 || nm < (int)nbk);
            const int fi = face_idx(a, x, y, z);
            if (fwd_any) div1 += pn[a];
            if (bwd_act) div1 -= crd[a] > 0 ? pn_own[a * 512 + t - kStride(a)] : hal_p[a * 192 + a * 64 + fi];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if (fwd_act)
                    div2[c] += crd[a] < 7 ? qn_own[qidx(a, c) * 512 + t + kStride(a)] : hal_q[qidx(a, c) * 192 + a * 64 + fi];
                if (bwd_any) div2[c] -= qn[qidx(a, c)];
            }
        }
        const float u0 = su[t];
        const float ut = u0 + A.tau * div1;
        // prox: generalised median = max_i min(ut - tau*lambda*W_i, c_i), c_n = +inf
        uint32_t hw[NP_MAX];
        float hsum = 0.0f;
#pragma unroll
        for (int k = 0; k < NP_MAX; ++k) {
            hw[k] = (NB || k < npairs) ? sh[k * 512 + t] : 0u;
            hsum += (float)(hw[k] & 0xffffu) + (float)(hw[k] >> 16);
        }
        float W = -hsum;
        float un = -INFINITY;
#pragma unroll
        for (int i = 0; i < NB_MAX; ++i) {
            if (NB || i < nbins) {
                const float hi = (float)((hw[i >> 1] >> ((i & 1) * 16)) & 0xffffu);
                un = fmaxf(un, fminf(ut - A.taulam * W, A.c[i]));
                W += 2.0f * hi;
            }
        }
        un = fmaxf(un, ut - A.taulam * W);
        if (A.clamp_u) un = fminf(1.0f, fmaxf(-1.0f, un));

        const size_t vi = (size_t)b * TGV_BVOX + t;
        A.u[vi] = un;
        A.ubar_out[vi] = 2.0f * un - u0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t oi = ((size_t)b * 3 + c) * TGV_BVOX + t;
            const float v0 = ld_s(sv + c * 512 + t);
            const float v1 = v0 + A.tau * (pn[c] + div2[c]);
            st_s(A.v + oi, v1);
            st_s(A.vbar_out + oi, 2.0f * v1 - v0);
            st_d(A.p_out + oi, pn[c], A.ds.isp);
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) st_d(A.q_out + ((size_t)b * 6 + c) * TGV_BVOX + t, qn[c], A.ds.isq);

        // ---- every thread is done with stage s: refill it with brick b + 2G
        __syncthreads();
        if (t == 0 && it + 2 * G < nit) {
            fence_proxy_async_smem();
            issue(s, brick(it + 2 * G));
        }
    }
    if (bail && t == 0) {
        atomicExch(P.err, 1);
        // copies may still be landing in either stage: wait for them (bounded) before leaving
        for (int k = 0; k < 2; ++k) {
            if (it + k * G < nit) mbar_wait_bounded(&bar[s ^ k], (parity >> (s ^ k)) & 1u, TGV_WAIT_CYCLES_DEFAULT);
        }
    }
}

namespace {

template <typename S, typename D, int NB>
tgv_status launch_pipe_t(tgv_domain* d, TgvLevel& L, int iters)
{
    const uint32_t SB = sizeof(S), SD = sizeof(D);
    const int npairs = (d->prm.nbins + 1) / 2;
    const uint32_t tx = 4096 + (6 * SB + 9 * SD) * 512 + npairs * 2048;
    const uint32_t stage = (tx + 127) / 128 * 128;
    uint32_t off = 2 * stage;
    PipeArgs<S, D> P;
    if (SD == 4) {
        P.off_pn = P.off_qn = 0;
    } else {
        P.off_pn = off;
        off += 3 * 512 * 4;
        P.off_qn = off;
        off += 6 * 512 * 4;
    }
    P.off_hp = off;
    off += 3 * 192 * 4;
    P.off_hq = off;
    off += 6 * 192 * 4;
    P.off_nbr = off;
    off += 2 * TGV_NNBR * 4;
    off = (off + 15) / 16 * 16;
    P.off_bar = off;
    off += 2 * 8;
    const size_t smem = off;
    auto kern = tgv_iter_pipe_kernel<S, D, NB>;
    int per_sm = 0;
    tgv_status st = tgv_kernel_setup((const void*)kern, TGV_BVOX, smem, &per_sm);
    if (st != TGV_OK) return tgv_fail(d, st, "pipe kernel setup (shared memory attribute / occupancy) failed");
    if (per_sm < 1) return tgv_fail(d, TGV_ERR_UNSUPPORTED, "pipe iteration kernel does not fit on an SM");
    int64_t grid = (int64_t)per_sm * d->sm_count;
    if (grid > tgv_work_items(L)) grid = tgv_work_items(L);
    P.err = d->err;
    P.wait_budget = tgv_wait_budget(d->prm);
    P.stage_bytes = stage;
    P.tx_bytes = tx;
    for (int it = 0; it < iters; ++it) {
        P.it = tgv_make_iter_args<S, D>(d, L);
        kern<<<(unsigned)grid, TGV_BVOX, smem, d->stream>>>(P);
        d->launches++;
        L.cur ^= 1;
    }
    return tgv_cuda_check(d, cudaGetLastError(), "tgv_iter_pipe_kernel launch");
}

template <typename S, typename D = S>
tgv_status launch_pipe_bins(tgv_domain* d, TgvLevel& L, int iters)
{
    switch (d->prm.nbins) {
    case 8: return launch_pipe_t<S, D, 8>(d, L, iters);
    case 10: return launch_pipe_t<S, D, 10>(d, L, iters);
    case 12: return launch_pipe_t<S, D, 12>(d, L, iters);
    default: return launch_pipe_t<S, D, 0>(d, L, iters);
    }
}

}  // namespace

// The pipelined kernels index with 64-bit offsets: every level qualifies.
bool tgv_pipe_supports(const TgvLevel& L) { return L.nb + L.nf < ((int64_t)1 << 31); }

tgv_status tgv_launch_iterations_pipe(tgv_domain* d, TgvLevel& L, int iters)
{
    if (tgv_work_items(L) == 0 || iters == 0) return TGV_OK;
    switch (d->prm.storage) {
    case TGV_STORAGE_FP32: return launch_pipe_bins<float>(d, L, iters);
    case TGV_STORAGE_BF16: return launch_pipe_bins<__nv_bfloat16>(d, L, iters);
    case TGV_STORAGE_FP16: return launch_pipe_bins<__half>(d, L, iters);
    case TGV_STORAGE_FX16: return launch_pipe_bins<__half, int16_t>(d, L, iters);
    }
    return tgv_fail(d, TGV_ERR_INVALID_ARG, "unknown storage type");
}
