// Fused TGV primal-dual iteration over 8^3 bricks, and the energy / gap
// reduction (Eq. 2-3; primal-dual method of Sec. 3.2).
//
// One CTA of 512 threads owns one active brick (one thread per voxel) and
// performs a whole iteration for it in a single pass over HBM:
//   phase A  new p, q at its own voxels from the old ubar/vbar/p/q;
//            new p on the three -face halo layers and new q on the three
//            +face halo layers are recomputed from the neighbours' old data
//            (the primal step needs them and another CTA owns them);
//   phase B  div1 p, div2 q from shared memory, histogram prox, clamp,
//            v update and over-relaxation; write u, v in place and
//            ubar, vbar, p, q to the other ping-pong copy.
// Traffic per voxel and iteration: read u, ubar, v, vbar, p, q, hist and write
// u, ubar, v, vbar, p, q once (halo re-reads hit L2).
#include <math.h>

#include <atomic>

#include "tgv_internal.cuh"

namespace {

__device__ __forceinline__ int face_index(int a, int x, int y, int z)
{
    return a == 0 ? y + 8 * z : (a == 1 ? x + 8 * z : x + 8 * y);
}

// Projections onto |p|_2 <= alpha and |q|_F <= alpha: scale by alpha/|.| when outside.
__device__ __forceinline__ void proj3(float p[3], float alpha)
{
    const float n2 = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
    if (n2 > alpha * alpha) {
        const float s = alpha * rsqrtf(n2);
        p[0] *= s;
        p[1] *= s;
        p[2] *= s;
    }
}

__device__ __forceinline__ void proj6(float q[6], float alpha)
{
    const float n2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + 2.0f * (q[3] * q[3] + q[4] * q[4] + q[5] * q[5]);
    if (n2 > alpha * alpha) {
        const float s = alpha * rsqrtf(n2);
#pragma unroll
        for (int c = 0; c < 6; ++c) q[c] *= s;
    }
}

// index of q_ab in the 6-component storage
__device__ __forceinline__ int qi(int a, int b)
{
    return a == b ? a : (a + b == 1 ? 3 : (a + b == 2 ? 4 : 5));
}

}  // namespace

template <typename S, typename D>
__global__ void __launch_bounds__(512, 2) tgv_iter_kernel(const IterArgs<S, D> A)
{
    __shared__ float s_ub[TGV_BVOX];
    __shared__ float s_vb[3][TGV_BVOX];
    __shared__ float s_p[3][TGV_BVOX + 192];
    __shared__ float s_q[6][TGV_BVOX + 192];
    __shared__ int s_nbr[TGV_NNBR];

    const int64_t b = A.work ? (int64_t)A.work[blockIdx.x] : (int64_t)blockIdx.x;
    const int t = threadIdx.x;
    const int x = t & 7, y = (t >> 3) & 7, z = t >> 6;
    const int crd[3] = {x, y, z};
    const int strd[3] = {1, 8, 64};

    if (t < TGV_NNBR) s_nbr[t] = A.nbr[b * TGV_NNBR + t];
    const float ub = A.ubar_in[b * TGV_BVOX + t];
    s_ub[t] = ub;
    float vb[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        vb[c] = ld_s(A.vbar_in + (b * 3 + c) * TGV_BVOX + t);
        s_vb[c][t] = vb[c];
    }
    __syncthreads();

    // ---------------- phase A: dual ascent + projection at the own voxel
    float pn[3], qn[6];
    {
        float g[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float nv = ub;  // "none" -> zero difference
            if (crd[a] < 7) {
                nv = s_ub[t + strd[a]];
            } else {
                int n = s_nbr[nb_plus(a)];
                if (n >= 0) nv = A.ubar_in[(int64_t)n * TGV_BVOX + t - 7 * strd[a]];
            }
            g[a] = nv - ub;
        }
        float dm[3][3];  // dm[a][c] = backward difference of vbar_c along a
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            int n = -2;
            if (crd[a] == 0) n = s_nbr[nb_minus(a)];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float w = vb[c];
                if (crd[a] > 0) w = s_vb[c][t - strd[a]];
                else if (n >= 0) w = ld_s(A.vbar_in + ((int64_t)n * 3 + c) * TGV_BVOX + t + 7 * strd[a]);
                dm[a][c] = vb[c] - w;
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) pn[c] = ld_d(A.p_in + (b * 3 + c) * TGV_BVOX + t, A.ds.dsp) + A.sigma * (g[c] - vb[c]);
        proj3(pn, A.alpha1);
        float e[6] = {dm[0][0], dm[1][1], dm[2][2], 0.5f * (dm[0][1] + dm[1][0]), 0.5f * (dm[0][2] + dm[2][0]),
                      0.5f * (dm[1][2] + dm[2][1])};
#pragma unroll
        for (int c = 0; c < 6; ++c) qn[c] = ld_d(A.q_in + (b * 6 + c) * TGV_BVOX + t, A.ds.dsq) + A.sigma * e[c];
        proj6(qn, A.alpha0);
#pragma unroll
        for (int c = 0; c < 3; ++c) s_p[c][t] = pn[c];
#pragma unroll
        for (int c = 0; c < 6; ++c) s_q[c][t] = qn[c];
    }

    // ---------------- phase A': halo duals owned by neighbouring bricks
    if (t < 192) {
        // new p on the -a face halo (voxel at coordinate -1 along a)
        const int a = t >> 6, k = t & 63;
        const int n = s_nbr[nb_minus(a)];
        if (n >= 0 && n < A.nb) {
            const int u0 = k & 7, u1 = k >> 3;  // the two face coordinates, lower axis first
            int hc[3];
            hc[a] = 7;
            hc[a == 0 ? 1 : 0] = u0;
            hc[a == 2 ? 1 : 2] = u1;
            const int lh = hc[0] + 8 * hc[1] + 64 * hc[2];
            const int lo = lh - 7 * strd[a];  // own voxel at coordinate 0 along a
            const float* ubn = A.ubar_in + (int64_t)n * TGV_BVOX;
            const float uh = ubn[lh];
            float g[3];
#pragma unroll
            for (int bb = 0; bb < 3; ++bb) {
                float nv = uh;
                if (bb == a) {
                    nv = s_ub[lo];
                } else if (hc[bb] < 7) {
                    nv = ubn[lh + strd[bb]];
                } else {
                    int e = s_nbr[nb_edge(a, bb)];
                    if (e >= 0) nv = A.ubar_in[(int64_t)e * TGV_BVOX + lh - 7 * strd[bb]];
                }
                g[bb] = nv - uh;
            }
            float ph[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float vh = ld_s(A.vbar_in + ((int64_t)n * 3 + c) * TGV_BVOX + lh);
                ph[c] = ld_d(A.p_in + ((int64_t)n * 3 + c) * TGV_BVOX + lh, A.ds.dsp) + A.sigma * (g[c] - vh);
            }
            proj3(ph, A.alpha1);
#pragma unroll
            for (int c = 0; c < 3; ++c) s_p[c][TGV_BVOX + a * 64 + k] = ph[c];
        }
    } else if (t < 384) {
        // new q on the +a face halo (voxel at coordinate 8 along a)
        const int tt = t - 192;
        const int a = tt >> 6, k = tt & 63;
        const int n = s_nbr[nb_plus(a)];
        if (n >= 0 && n < A.nb) {
            const int u0 = k & 7, u1 = k >> 3;
            int hc[3];
            hc[a] = 0;
            hc[a == 0 ? 1 : 0] = u0;
            hc[a == 2 ? 1 : 2] = u1;
            const int lh = hc[0] + 8 * hc[1] + 64 * hc[2];
            const int lo = lh + 7 * strd[a];  // own voxel at coordinate 7 along a
            float vh[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) vh[c] = ld_s(A.vbar_in + ((int64_t)n * 3 + c) * TGV_BVOX + lh);
            float dm[3][3];
#pragma unroll
            for (int bb = 0; bb < 3; ++bb) {
                int src = -1;  // brick to read from, -1: none
                int li = 0;
                bool own = false;
                if (bb == a) {
                    own = true;
                } else if (hc[bb] > 0) {
                    src = n;
                    li = lh - strd[bb];
                } else {
                    src = s_nbr[nb_edge(bb, a)];  // offset +1 along a, -1 along bb
                    li = lh + 7 * strd[bb];
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float w = vh[c];
                    if (own) w = s_vb[c][lo];
                    else if (src >= 0) w = ld_s(A.vbar_in + ((int64_t)src * 3 + c) * TGV_BVOX + li);
                    dm[bb][c] = vh[c] - w;
                }
            }
            float e[6] = {dm[0][0], dm[1][1], dm[2][2], 0.5f * (dm[0][1] + dm[1][0]), 0.5f * (dm[0][2] + dm[2][0]),
                          0.5f * (dm[1][2] + dm[2][1])};
            float qh[6];
#pragma unroll
            for (int c = 0; c < 6; ++c)
                qh[c] = ld_d(A.q_in + ((int64_t)n * 6 + c) * TGV_BVOX + lh, A.ds.dsq) + A.sigma * e[c];
            proj6(qh, A.alpha0);
#pragma unroll
            for (int c = 0; c < 6; ++c) s_q[c][TGV_BVOX + a * 64 + k] = qh[c];
        }
    }
    __syncthreads();

    // ---------------- phase B: primal descent, prox, over-relaxation
    float div1 = 0.0f;
    float div2[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int np = crd[a] < 7 ? 0 : s_nbr[nb_plus(a)];   // >= 0: forward exists (same brick = 0)
        const int nm = crd[a] > 0 ? 0 : s_nbr[nb_minus(a)];  // >= 0: backward exists
        const bool fwd_any = np >= 0;
        const bool fwd_act = np >= 0 && (crd[a] < 7 || np < A.nb);
        const bool bwd_any = nm >= 0;
        const bool bwd_act = nm >= 0 && (crd[a] > 0 || nm < A.nb);
        if (fwd_any) div1 += pn[a];
        if (bwd_act) div1 -= crd[a] > 0 ? s_p[a][t - strd[a]] : s_p[a][TGV_BVOX + a * 64 + face_index(a, x, y, z)];
        const int fi = crd[a] < 7 ? t + strd[a] : TGV_BVOX + a * 64 + face_index(a, x, y, z);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (fwd_act) div2[c] += s_q[qi(a, c)][fi];
            if (bwd_any) div2[c] -= qn[qi(a, c)];
        }
    }

    const int64_t vi = b * TGV_BVOX + t;
    const float u0 = A.u[vi];
    const float ut = u0 + A.tau * div1;
    // prox of tau*lambda*sum_b h_b|u - c_b|: the generalised median of
    // {c_b} and {ut - tau*lambda*W_i}, W_i = sum_{b<i} h_b - sum_{b>=i} h_b.
    // With c ascending and the W_i ascending, the median equals
    // max_i min(ut - tau*lambda*W_i, c_i) (c_n = +inf).
    float hsum = 0.0f;
    uint32_t hw[TGV_MAX_BINS / 2];
#pragma unroll
    for (int k = 0; k < TGV_MAX_BINS / 2; ++k) {
        hw[k] = k < A.npairs ? A.hist[((int64_t)b * A.npairs + k) * TGV_BVOX + t] : 0u;
        hsum += (float)(hw[k] & 0xffffu) + (float)(hw[k] >> 16);
    }
    float W = -hsum;
    float un = -INFINITY;
#pragma unroll
    for (int i = 0; i < TGV_MAX_BINS; ++i) {
        if (i < A.nbins) {
            const float hi = (float)((hw[i >> 1] >> ((i & 1) * 16)) & 0xffffu);
            un = fmaxf(un, fminf(ut - A.taulam * W, A.c[i]));
            W += 2.0f * hi;
        }
    }
    un = fmaxf(un, ut - A.taulam * W);
    if (A.clamp_u) un = fminf(1.0f, fmaxf(-1.0f, un));

    A.u[vi] = un;
    A.ubar_out[vi] = 2.0f * un - u0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int64_t oi = (b * 3 + c) * TGV_BVOX + t;
        const float v0 = ld_s(A.v + oi);
        const float v1 = v0 + A.tau * (pn[c] + div2[c]);
        st_s(A.v + oi, v1);
        st_s(A.vbar_out + oi, 2.0f * v1 - v0);
        st_d(A.p_out + oi, pn[c], A.ds.isp);
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) st_d(A.q_out + (b * 6 + c) * TGV_BVOX + t, qn[c], A.ds.isq);
}

// =====================================================================================
// Energy, dual value and gap (FP32 per-voxel terms, FP64 accumulation,
// fixed-order reduction: per-block partials, then one block sums them in order).
// =====================================================================================
template <typename S, typename D>
struct EnergyArgs {
    const float* u;
    const S* v;
    const D* p;
    const D* q;
    float dsp, dsq;  // fixed-point decode scales of p and q (TGV_STORAGE_FX16)
    const uint32_t* hist;
    const int32_t* nbr;
    const int32_t* work;  // item -> brick (nullptr: identity)
    int64_t nb, nall, nitems;
    int nbins, npairs;
    float alpha1, alpha0, lambda, box_v;
    float c[TGV_MAX_BINS];
    double* partial;  // [gridDim.x][3]: energy, dual, max|v|
};

namespace {

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

}  // namespace

// Persistent CTAs of 64 threads, sixteen per SM, taking bricks in turn; a thread
// evaluates eight voxels of a brick, one z layer per round (64 registers, no
// spills: fewer threads with more voxels each hide the load latency better than
// one voxel per thread -- at 256^3, 466 us against 586 us for 512 threads per
// brick at three CTAs per SM).  NB: bin count as a compile-time constant (8, 10,
// 12), 0 = read at run time.  Own fields through per-brick base pointers;
// neighbours in the same brick or across a face.
template <typename S, typename D, int NB>
__global__ void __launch_bounds__(64, 16) tgv_energy_kernel(const EnergyArgs<S, D> A)
{
    constexpr int NBM = NB ? NB : TGV_MAX_BINS;
    __shared__ int32_t s_nbr2[2][TGV_NNBR];
    __shared__ double s_red[3][16];
    const int tid = threadIdx.x;  // voxels tid + 64 k (k = 0..7) of each brick
    auto brick_of = [&](int64_t i) -> int64_t { return A.work ? (int64_t)A.work[i] : i; };
    // neighbour rows double-buffered: the next brick's row is loaded while this one
    // is evaluated and stored before the barrier that opens the next brick
    if (tid < TGV_NNBR && (int64_t)blockIdx.x < A.nitems) s_nbr2[0][tid] = A.nbr[brick_of(blockIdx.x) * TGV_NNBR + tid];
    int buf = 0;
    // per-warp running sums over the CTA's bricks (FP64, in brick order)
    double acc_en = 0.0, acc_du = 0.0, acc_vm = 0.0;
    for (int64_t item = blockIdx.x; item < A.nitems; item += gridDim.x, buf ^= 1) {
    const int64_t b = brick_of(item);
    const int64_t nx = item + gridDim.x;
    int32_t nbr_next = 0;
    if (tid < TGV_NNBR && nx < A.nitems) nbr_next = A.nbr[brick_of(nx) * TGV_NNBR + tid];
    __syncthreads();  // this brick's row is in place; the other buffer is no longer read
    const int32_t* s_nbr = s_nbr2[buf];
    const int nbins = NB ? NB : A.nbins;
    float en_t = 0.0f, du_t = 0.0f, vm_t = 0.0f;
    for (int half = 0; half < 8; ++half) {
    const int t = tid + 64 * half;
    const int crd[3] = {t & 7, (t >> 3) & 7, t >> 6};
    const float* ub = A.u + b * TGV_BVOX;
    const S* vb = A.v + b * 3 * TGV_BVOX;
    const D* pb = A.p + b * 3 * TGV_BVOX;
    const D* qb = A.q + b * 6 * TGV_BVOX;
    const float u = ub[t];
    float v[3], p[3], q[6];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        v[c] = ld_s(vb + c * TGV_BVOX + t);
        p[c] = ld_d(pb + c * TGV_BVOX + t, A.dsp);
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) q[c] = ld_d(qb + c * TGV_BVOX + t, A.dsq);

    float gmv2 = 0.0f, k0 = 0.0f, dm[3][3], dk[3][3], div1 = 0.0f, div2[3] = {0, 0, 0};
    float vmax = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int strd = a == 0 ? 1 : (a == 1 ? 8 : 64);
        vmax = fmaxf(vmax, fabsf(v[a]));
        // forward neighbour: brick nf (-1 none), local index lf
        int64_t nf = b, nbk = b;
        int lf = t + strd, lb = t - strd;
        if (crd[a] == 7) {
            nf = s_nbr[nb_plus(a)];
            lf = t - 7 * strd;
        }
        if (crd[a] == 0) {
            nbk = s_nbr[nb_minus(a)];
            lb = t + 7 * strd;
        }
        // forward gradient of u (frozen neighbours give their constant)
        float g = 0.0f;
        if (nf >= 0) {
            const float un = A.u[nf * TGV_BVOX + lf];
            g = un - u;
            if (nf >= A.nb) k0 += un * p[a];  // frozen constant paired with p
        }
        const float d = g - v[a];
        gmv2 += d * d;
        // backward differences of v
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            dm[a][c] = 0.0f;
            dk[a][c] = 0.0f;
        }
        if (nbk >= 0) {
            const S* vn = A.v + nbk * 3 * TGV_BVOX + lb;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float w = ld_s(vn + c * TGV_BVOX);
                dm[a][c] = v[c] - w;
                if (nbk >= A.nb) dk[a][c] = -w;  // frozen constant part of E(v)
            }
        }
        // div1 p and div2 q
        if (nf >= 0) div1 += p[a];
        if (nbk >= 0 && nbk < A.nb) div1 -= ld_d(A.p + (nbk * 3 + a) * TGV_BVOX + lb, A.dsp);
        const bool qact = nf >= 0 && nf < A.nb;
        const D* qn = A.q + (qact ? nf * 6 * TGV_BVOX + lf : 0);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (qact) div2[c] += ld_d(qn + qi(a, c) * TGV_BVOX, A.dsq);
            if (nbk >= 0) div2[c] -= q[qi(a, c)];
        }
    }
    const float e[6] = {dm[0][0], dm[1][1], dm[2][2], 0.5f * (dm[0][1] + dm[1][0]), 0.5f * (dm[0][2] + dm[2][0]),
                        0.5f * (dm[1][2] + dm[2][1])};
    const float ek[6] = {dk[0][0], dk[1][1], dk[2][2], 0.5f * (dk[0][1] + dk[1][0]), 0.5f * (dk[0][2] + dk[2][0]),
                         0.5f * (dk[1][2] + dk[2][1])};
    float ef2 = e[0] * e[0] + e[1] * e[1] + e[2] * e[2] + 2.0f * (e[3] * e[3] + e[4] * e[4] + e[5] * e[5]);
    k0 += ek[0] * q[0] + ek[1] * q[1] + ek[2] * q[2] + 2.0f * (ek[3] * q[3] + ek[4] * q[4] + ek[5] * q[5]);

    // data term lambda*sum_b h_b|u - c_b| at u, and its conjugate phi*(div1 p): the
    // maximum of w*u - data(u) over the breakpoints {-1, c_0..c_{n-1}, +1}.  With
    // prefix sums H_< , S_< (counts and count-weighted centres below bin k):
    //   data(c_k) = lambda (c_k (H_< - H_>) - (S_< - S_>)).
    uint32_t hw[(NBM + 1) / 2];
    const uint32_t* hb0 = A.hist + (int64_t)b * ((nbins + 1) / 2) * TGV_BVOX + t;
#pragma unroll
    for (int k = 0; k < (NBM + 1) / 2; ++k) hw[k] = (NB || 2 * k < nbins) ? hb0[k * TGV_BVOX] : 0u;
    float hb[NBM];
    float H = 0.0f, Sc = 0.0f, du_own = 0.0f;
#pragma unroll
    for (int k = 0; k < NBM; ++k) {
        hb[k] = 0.0f;
        if (NB || k < nbins) {
            // count k as a float: its 16 bits as the mantissa of 2^23 (a byte permute),
            // minus 2^23 (exact), instead of an integer conversion
            const uint32_t sel = (k & 1) ? 0x7632u : 0x7610u;
            hb[k] = __uint_as_float(__byte_perm(hw[k >> 1], 0x4B000000u, sel)) - 8388608.0f;
            H += hb[k];
            Sc += hb[k] * A.c[k];
            du_own += hb[k] * fabsf(u - A.c[k]);
        }
    }
    float best = fmaxf(-div1 - A.lambda * (Sc + H), div1 - A.lambda * (H - Sc));
    {
        // at breakpoint c_k, with H_< , S_< the counts and count-weighted centres below bin
        // k: c_k (H_< - H_>) - (S_< - S_>) = c_k (2 H_< - H) - (2 S_< - S) (the bin's own
        // h_k c_k cancels), so with A = 2 H_< - H and B = S - 2 S_<, updated bin by bin:
        // div1 c_k - data(c_k) = c_k (div1 - lambda A) - lambda B
        float Ak = -H, Bk = Sc;
#pragma unroll
        for (int k = 0; k < NBM; ++k) {
            if (NB || k < nbins) {
                best = fmaxf(best, A.c[k] * (div1 - A.lambda * Ak) - A.lambda * Bk);
                Ak += 2.0f * hb[k];
                Bk -= 2.0f * hb[k] * A.c[k];
            }
        }
    }
    float l1 = fabsf(p[0] + div2[0]) + fabsf(p[1] + div2[1]) + fabsf(p[2] + div2[2]);

    // per-voxel terms in FP32; warps reduce in FP32 (tree of 32: relative error
    // below 5 ulp), warps and blocks in FP64, all in a fixed order
    en_t += A.alpha1 * sqrtf(gmv2) + A.alpha0 * sqrtf(ef2) + A.lambda * du_own;
    du_t += k0 - best - A.box_v * l1;
    vm_t = fmaxf(vm_t, vmax);
    }
    float en = en_t, du = du_t, vm = vm_t;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        en += __shfl_down_sync(0xffffffffu, en, o);
        du += __shfl_down_sync(0xffffffffu, du, o);
        vm = fmaxf(vm, __shfl_down_sync(0xffffffffu, vm, o));
    }
    acc_en += (double)en;
    acc_du += (double)du;
    acc_vm = fmax(acc_vm, (double)vm);
    if (tid < TGV_NNBR && nx < A.nitems) s_nbr2[buf ^ 1][tid] = nbr_next;
    }
    const int w = tid >> 5, lane = tid & 31;
    if (lane == 0) {
        s_red[0][w] = acc_en;
        s_red[1][w] = acc_du;
        s_red[2][w] = acc_vm;
    }
    __syncthreads();
    if (tid == 0) {
        double se = 0.0, sd = 0.0, sm = 0.0;
        for (int k = 0; k < (int)blockDim.x / 32; ++k) {
            se += s_red[0][k];
            sd += s_red[1][k];
            sm = fmax(sm, s_red[2][k]);
        }
        A.partial[3 * blockIdx.x + 0] = se;
        A.partial[3 * blockIdx.x + 1] = sd;
        A.partial[3 * blockIdx.x + 2] = sm;
    }
}

// CTAs of the persistent energy kernel: sixteen per SM (capped by the bricks)
int64_t tgv_energy_grid(int64_t nitems)
{
    // SM count of the current device, cached per device (threads may race to fill an
    // entry; they all store the same value)
    static std::atomic<int> sms[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    int n = sms[dev].load(std::memory_order_relaxed);
    if (n <= 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
        sms[dev].store(n, std::memory_order_relaxed);
    }
    const int64_t g = 16 * (int64_t)n;
    return nitems < g ? nitems : g;
}

// launches the energy kernel; returns its grid (the number of partials)
template <typename S, typename D>
static int64_t launch_energy_kernel(EnergyArgs<S, D> A, int64_t nitems, cudaStream_t stream)
{
    const int64_t grid = tgv_energy_grid(nitems);
    A.nitems = nitems;
    switch (A.nbins) {
    case 8: tgv_energy_kernel<S, D, 8><<<(unsigned)grid, 64, 0, stream>>>(A); break;
    case 10: tgv_energy_kernel<S, D, 10><<<(unsigned)grid, 64, 0, stream>>>(A); break;
    case 12: tgv_energy_kernel<S, D, 12><<<(unsigned)grid, 64, 0, stream>>>(A); break;
    default: tgv_energy_kernel<S, D, 0><<<(unsigned)grid, 64, 0, stream>>>(A); break;
    }
    return grid;
}

// One block sums the per-block partials in a fixed order.
__global__ void __launch_bounds__(1024) tgv_reduce_partials(const double* partial, int64_t n, float box_v, double* out)
{
    __shared__ double s[3][32];
    const int t = threadIdx.x;
    double en = 0.0, du = 0.0, vm = 0.0;
    for (int64_t i = t; i < n; i += blockDim.x) {
        en += partial[3 * i];
        du += partial[3 * i + 1];
        vm = fmax(vm, partial[3 * i + 2]);
    }
    en = warp_sum(en);
    du = warp_sum(du);
    vm = warp_max(vm);
    const int w = t >> 5, lane = t & 31;
    if (lane == 0) {
        s[0][w] = en;
        s[1][w] = du;
        s[2][w] = vm;
    }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        en = lane < nw ? s[0][lane] : 0.0;
        du = lane < nw ? s[1][lane] : 0.0;
        vm = lane < nw ? s[2][lane] : 0.0;
        en = warp_sum(en);
        du = warp_sum(du);
        vm = warp_max(vm);
        if (lane == 0) {
            out[0] = en;
            out[1] = du;
            out[2] = en - du;
            out[3] = vm <= (double)box_v ? 1.0 : 0.0;
        }
    }
}

// =====================================================================================
// host launchers
// =====================================================================================
template <typename S, typename D = S>
static tgv_status launch_iters_t(tgv_domain* d, TgvLevel& L, int iters)
{
    for (int it = 0; it < iters; ++it) {
        IterArgs<S, D> A = tgv_make_iter_args<S, D>(d, L);
        tgv_iter_kernel<S, D><<<(unsigned)A.nitems, TGV_BVOX, 0, d->stream>>>(A);
        d->launches++;
        L.cur ^= 1;
    }
    return tgv_cuda_check(d, cudaGetLastError(), "tgv_iter_kernel launch");
}

tgv_status tgv_launch_iterations(tgv_domain* d, TgvLevel& L, int iters)
{
    if (tgv_work_items(L) == 0 || iters == 0) return TGV_OK;
    if (d->prm.iter_kernel == TGV_ITER_PAIRED && tgv_pipe_supports(L)) return tgv_launch_iterations_pair(d, L, iters);
    if (d->prm.iter_kernel == TGV_ITER_PIPELINED && tgv_pipe_supports(L)) return tgv_launch_iterations_pipe(d, L, iters);
    switch (d->prm.storage) {
    case TGV_STORAGE_FP32: return launch_iters_t<float>(d, L, iters);
    case TGV_STORAGE_BF16: return launch_iters_t<__nv_bfloat16>(d, L, iters);
    case TGV_STORAGE_FP16: return launch_iters_t<__half>(d, L, iters);
    case TGV_STORAGE_FX16: return launch_iters_t<__half, int16_t>(d, L, iters);
    }
    return tgv_fail(d, TGV_ERR_INVALID_ARG, "unknown storage type");
}

template <typename S, typename D = S>
static tgv_status launch_energy_t(tgv_domain* d, TgvLevel& L, double* host_out)
{
    const int64_t nitems = tgv_work_items(L);
    tgv_status st = tgv_scratch(d, d->red, sizeof(double) * 3 * (size_t)nitems);
    if (st != TGV_OK) return st;
    EnergyArgs<S, D> A;
    A.u = L.u;
    A.v = (const S*)L.v;
    A.p = (const D*)L.p[L.cur];
    A.q = (const D*)L.q[L.cur];
    const DualScales ds = tgv_dual_scales(d->prm);
    A.dsp = ds.dsp;
    A.dsq = ds.dsq;
    A.hist = L.hist;
    A.nbr = L.nbr;
    A.work = L.work;
    A.nb = L.nb;
    A.nall = L.nb + L.nf;
    A.nbins = d->prm.nbins;
    A.npairs = (d->prm.nbins + 1) / 2;
    A.alpha1 = d->prm.alpha1;
    A.alpha0 = d->prm.alpha0;
    A.lambda = d->prm.lambda;
    A.box_v = d->prm.box_v;
    tgv_bin_centres(d->prm, A.c);
    A.partial = (double*)d->red.ptr;
    const int64_t parts = launch_energy_kernel<S, D>(A, nitems, d->stream);
    tgv_reduce_partials<<<1, 1024, 0, d->stream>>>(A.partial, parts, d->prm.box_v, d->red_out);
    d->launches += 2;
    st = tgv_cuda_check(d, cudaGetLastError(), "tgv_energy_kernel launch");
    if (st != TGV_OK) return st;
    st = tgv_cuda_check(d, cudaMemcpyAsync(host_out, d->red_out, 4 * sizeof(double), cudaMemcpyDeviceToHost, d->stream),
                        "energy copy");
    if (st != TGV_OK) return st;
    st = tgv_cuda_check(d, cudaStreamSynchronize(d->stream), "energy sync");
    if (st != TGV_OK) return st;
    return tgv_check_device_error(d);
}

tgv_status tgv_launch_energy(tgv_domain* d, TgvLevel& L, double* host_out)
{
    if (tgv_work_items(L) == 0) {
        for (int k = 0; k < 4; ++k) host_out[k] = k == 3 ? 1.0 : 0.0;
        return TGV_OK;
    }
    switch (d->prm.storage) {
    case TGV_STORAGE_FP32: return launch_energy_t<float>(d, L, host_out);
    case TGV_STORAGE_BF16: return launch_energy_t<__nv_bfloat16>(d, L, host_out);
    case TGV_STORAGE_FP16: return launch_energy_t<__half>(d, L, host_out);
    case TGV_STORAGE_FX16: return launch_energy_t<__half, int16_t>(d, L, host_out);
    }
    return tgv_fail(d, TGV_ERR_INVALID_ARG, "unknown storage type");
}

// Energy of a caller-described state with caller-given scratch: `partial`
// holds 3 doubles per active brick, `result` 4 doubles.  Launches the same two
// kernels as tgv_launch_energy on `stream`; no allocation, no synchronisation.
template <typename S, typename D = S>
static cudaError_t launch_energy_view_t(const tgv_state_view& s, const tgv_params& prm, cudaStream_t stream,
                                       double* partial, double* result)
{
    EnergyArgs<S, D> A;
    A.u = s.u;
    A.v = (const S*)s.v;
    A.p = (const D*)s.p;
    A.q = (const D*)s.q;
    const DualScales ds = tgv_dual_scales(prm);
    A.dsp = ds.dsp;
    A.dsq = ds.dsq;
    A.hist = s.hist;
    A.nbr = s.nbr;
    A.work = nullptr;
    A.nb = s.nbricks;
    A.nall = s.nall;
    A.nbins = prm.nbins;
    A.npairs = (prm.nbins + 1) / 2;
    A.alpha1 = prm.alpha1;
    A.alpha0 = prm.alpha0;
    A.lambda = prm.lambda;
    A.box_v = prm.box_v;
    tgv_bin_centres(prm, A.c);
    A.partial = partial;
    const int64_t parts = launch_energy_kernel<S, D>(A, s.nbricks, stream);
    tgv_reduce_partials<<<1, 1024, 0, stream>>>(partial, parts, prm.box_v, result);
    return cudaGetLastError();
}

cudaError_t tgv_launch_energy_view(const tgv_state_view& s, const tgv_params& prm, cudaStream_t stream,
                                   double* partial, double* result)
{
    switch (prm.storage) {
    case TGV_STORAGE_FP32: return launch_energy_view_t<float>(s, prm, stream, partial, result);
    case TGV_STORAGE_BF16: return launch_energy_view_t<__nv_bfloat16>(s, prm, stream, partial, result);
    case TGV_STORAGE_FX16: return launch_energy_view_t<__half, int16_t>(s, prm, stream, partial, result);
    default: return launch_energy_view_t<__half>(s, prm, stream, partial, result);
    }
}
