// The paired form's per-CTA machinery (Eq. 2-3, Sec. 3.2): a CTA streams whole bricks
// through shared memory with bulk asynchronous copies and, per brick, computes the new
// duals (phase A) and the primal step (phase B).  Shared by the level kernel
// (tgv_iter_pair.cu: strided runs of items over a level) and the persistent batched
// kernel (tgv_batched.cu: runs drawn from a ticket counter across many chunks).
#pragma once

#include <math.h>

#include <type_traits>

#include "tgv_async.cuh"
#include "tgv_internal.cuh"

namespace {

constexpr int kThreads = 256;

// ---------------------------------------------------------------- paired storage access
template <typename S> struct Pair;
template <> struct Pair<float> {
    using T = float2;
    static __device__ __forceinline__ float2 ld(const float* p) { return *(const float2*)p; }
    static __device__ __forceinline__ void st(float* p, float2 v) { *(float2*)p = v; }
};
template <> struct Pair<__nv_bfloat16> {
    static __device__ __forceinline__ float2 ld(const __nv_bfloat16* p)
    {
        return __bfloat1622float2(*(const __nv_bfloat162*)p);
    }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, float2 v)
    {
        *(__nv_bfloat162*)p = __floats2bfloat162_rn(v.x, v.y);
    }
};
template <> struct Pair<__half> {
    static __device__ __forceinline__ float2 ld(const __half* p) { return __half22float2(*(const __half2*)p); }
    static __device__ __forceinline__ void st(__half* p, float2 v) { *(__half2*)p = __floats2half2_rn(v.x, v.y); }
};

// ---------------------------------------------------------------- packed FP32 pairs
// The two voxels of a thread's pair go through the same operations.  sm_100 and later
// issue such a pair as one packed instruction (add / sub / mul / fma .rn.f32x2), each
// lane rounded exactly as the scalar operation, so a value computed in packed form has
// the same bits as the scalar form of the same operations (which the single-voxel halo
// tasks use).  Unlike the scalar __fmul_rn / __fadd_rn, a packed product that feeds a
// packed sum may still be fused into one multiply-add by the compiler, whatever the
// rounding modifier: code that must give the same bits on every path (the rounding of a
// new dual, phase B's sums of decoded duals) therefore never feeds a packed product into
// a packed sum.
#define TGV_F32X2_OP(name, op)                                                                  \
    __device__ __forceinline__ float2 name(float2 a, float2 b)                                  \
    {                                                                                           \
        float2 d;                                                                               \
        asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t" op \
            " rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"                                      \
            : "=f"(d.x), "=f"(d.y)                                                              \
            : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));                                         \
        return d;                                                                               \
    }
TGV_F32X2_OP(add2, "add.rn.f32x2")
TGV_F32X2_OP(sub2, "sub.rn.f32x2")
TGV_F32X2_OP(mul2, "mul.rn.f32x2")
#undef TGV_F32X2_OP
// a * b + c, rounded once
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c)
{
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mov.b64 rc, {%6, %7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
__device__ __forceinline__ float2 bc2(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 zero2() { return make_float2(0.0f, 0.0f); }

// pairs of dual values (p, q): the storage type's pair, or two 16-bit fixed-point values
// in one 32-bit word (TGV_STORAGE_FX16; sc = the decode or encode scale)
template <typename D> struct DPair {
    static __device__ __forceinline__ float2 ld(const D* p, float /*dsc*/) { return Pair<D>::ld(p); }
    static __device__ __forceinline__ void st(D* p, float2 v, float /*isc*/) { Pair<D>::st(p, v); }
};
template <> struct DPair<int16_t> {
    static __device__ __forceinline__ float2 ld(const int16_t* p, float dsc)
    {
        const uint32_t w = *(const uint32_t*)p;
        return make_float2(fx16_decode((int16_t)(w & 0xffffu), dsc), fx16_decode((int16_t)(w >> 16), dsc));
    }
    static __device__ __forceinline__ void st(int16_t* p, float2 v, float isc)
    {
        *(uint32_t*)p = fx16_encode2(v.x, v.y, isc);
    }
};

// A new dual as the level stores it.  16-bit duals are rounded to their storage type once,
// right after the projection, and that stored value is what the primal step, the run
// hand-overs and the recomputed halo duals use (so a brick's own new duals can live in its
// stage, in place of the old ones); FP32 duals are unchanged.
template <typename D> struct DRound {
    static __device__ __forceinline__ float r(float x, float /*dsc*/, float /*isc*/) { return x; }
};
template <> struct DRound<__half> {
    static __device__ __forceinline__ float r(float x, float, float) { return __half2float(__float2half_rn(x)); }
};
template <> struct DRound<__nv_bfloat16> {
    static __device__ __forceinline__ float r(float x, float, float)
    {
        return __bfloat162float(__float2bfloat16_rn(x));
    }
};
// Fixed point: x * isc + 1.5 * 2^23 in one fused operation (|x * isc| <= 32768 < 2^22 for a
// projected dual) rounds x * isc to the nearest integer k (ties to even), and k sits in the
// low bits of the sum; k * dsc is the stored value.  One rounding of the exact product,
// written as a fused multiply-add on every path (scalar, packed, store), so no compiler
// choice between a separate product and a fused one can make two paths differ.
constexpr float kRoundMagic = 12582912.0f;
template <> struct DRound<int16_t> {
    static __device__ __forceinline__ float r(float x, float dsc, float isc)
    {
        return __fmul_rn(__fsub_rn(__fmaf_rn(x, isc, kRoundMagic), kRoundMagic), dsc);
    }
};
// DRound of a pair (the same operations lane by lane)
template <typename D> struct DRound2 {
    static __device__ __forceinline__ float2 r(float2 v, float dsc, float isc)
    {
        return make_float2(DRound<D>::r(v.x, dsc, isc), DRound<D>::r(v.y, dsc, isc));
    }
};
template <> struct DRound2<float> {
    static __device__ __forceinline__ float2 r(float2 v, float, float) { return v; }
};
template <> struct DRound2<int16_t> {
    static __device__ __forceinline__ float2 r(float2 v, float dsc, float isc)
    {
        const float2 m = bc2(kRoundMagic);
        return mul2(sub2(fma2(v, bc2(isc), m), m), bc2(dsc));
    }
};

// Stores a pair of new duals in the storage type and replaces them by the stored values.
template <typename D> struct DRoundStore;
template <> struct DRoundStore<float> {
    static __device__ __forceinline__ void st(float* p, float2& v, float, float) { *(float2*)p = v; }
};
template <> struct DRoundStore<__half> {
    static __device__ __forceinline__ void st(__half* p, float2& v, float, float)
    {
        const __half2 h = __floats2half2_rn(v.x, v.y);
        *(__half2*)p = h;
        v = __half22float2(h);
    }
};
template <> struct DRoundStore<__nv_bfloat16> {
    static __device__ __forceinline__ void st(__nv_bfloat16* p, float2& v, float, float)
    {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
        *(__nv_bfloat162*)p = h;
        v = __bfloat1622float2(h);
    }
};
template <> struct DRoundStore<int16_t> {
    static __device__ __forceinline__ void st(int16_t* p, float2& v, float dsc, float isc)
    {
        const float2 m = bc2(kRoundMagic);
        const float2 s = fma2(v, bc2(isc), m);
        *(uint32_t*)p = __byte_perm(__float_as_uint(s.x), __float_as_uint(s.y), 0x5410);  // low halves: k_a, k_b
        v = mul2(sub2(s, m), bc2(dsc));
    }
};

// FX16 duals in units of their fixed-point step (the stored integer k itself): loads are
// integer-to-float conversions, and a new dual is rounded to the nearest integer by adding
// and subtracting 1.5 * 2^23 (|k| <= 32767.5 after a projection onto radius 32767).  The
// packed rounding adds through a fused multiply by 1, so no compiler fusion with the
// projection's product can change it.
__device__ __forceinline__ float2 fxk_ld2(const int16_t* p)
{
    const uint32_t w = *(const uint32_t*)p;
    return make_float2((float)(int16_t)(w & 0xffffu), (float)(int16_t)(w >> 16));
}
__device__ __forceinline__ float fxk_round(float x) { return __fsub_rn(__fadd_rn(x, kRoundMagic), kRoundMagic); }
__device__ __forceinline__ float2 fxk_round2(float2 v)
{
    const float2 m = bc2(kRoundMagic);
    return sub2(fma2(v, bc2(1.0f), m), m);
}
// stores the rounded pair (its low 16 bits) and returns it
__device__ __forceinline__ float2 fxk_store2(int16_t* p, float2 v)
{
    const float2 m = bc2(kRoundMagic);
    const float2 r = fma2(v, bc2(1.0f), m);
    *(uint32_t*)p = __byte_perm(__float_as_uint(r.x), __float_as_uint(r.y), 0x5410);
    return sub2(r, m);
}

__device__ __forceinline__ float2 ldf2(const float* p) { return *(const float2*)p; }
__device__ __forceinline__ void stf2(float* p, float2 v) { *(float2*)p = v; }

__device__ __forceinline__ int qidx(int a, int b) { return a == b ? a : (a + b == 1 ? 3 : (a + b == 2 ? 4 : 5)); }

// Dual updates of one voxel, every operation rounded explicitly (no contraction
// choices left to the compiler): the owner of a voxel and a neighbour that
// recomputes it as a halo get the same bits from the same inputs.
// p <- proj_{|.| <= alpha1}(p + sigma (g - vb)),  g = grad ubar, vb = vbar
__device__ __forceinline__ void upd_p(float p[3], const float g[3], const float vb[3], float sigma, float alpha1,
                                      float a1sq)
{
#pragma unroll
    for (int c = 0; c < 3; ++c) p[c] = __fmaf_rn(sigma, __fsub_rn(g[c], vb[c]), p[c]);
    const float n2 = __fmaf_rn(p[2], p[2], __fmaf_rn(p[1], p[1], __fmul_rn(p[0], p[0])));
    if (n2 > a1sq) {
        const float s = __fmul_rn(alpha1, rsqrtf(n2));
#pragma unroll
        for (int c = 0; c < 3; ++c) p[c] = __fmul_rn(p[c], s);
    }
}

// q <- proj_{|.|_F <= alpha0}(q + sigma E(vbar)); dm[a][c] = backward difference of vbar_c along a
__device__ __forceinline__ void upd_q(float q[6], const float dm[3][3], float sigma, float alpha0, float a0sq)
{
    q[0] = __fmaf_rn(sigma, dm[0][0], q[0]);
    q[1] = __fmaf_rn(sigma, dm[1][1], q[1]);
    q[2] = __fmaf_rn(sigma, dm[2][2], q[2]);
    q[3] = __fmaf_rn(sigma, __fmul_rn(0.5f, __fadd_rn(dm[0][1], dm[1][0])), q[3]);
    q[4] = __fmaf_rn(sigma, __fmul_rn(0.5f, __fadd_rn(dm[0][2], dm[2][0])), q[4]);
    q[5] = __fmaf_rn(sigma, __fmul_rn(0.5f, __fadd_rn(dm[1][2], dm[2][1])), q[5]);
    const float off = __fmaf_rn(q[5], q[5], __fmaf_rn(q[4], q[4], __fmul_rn(q[3], q[3])));
    const float n2 = __fmaf_rn(2.0f, off, __fmaf_rn(q[2], q[2], __fmaf_rn(q[1], q[1], __fmul_rn(q[0], q[0]))));
    if (n2 > a0sq) {
        const float s = __fmul_rn(alpha0, rsqrtf(n2));
#pragma unroll
        for (int c = 0; c < 6; ++c) q[c] = __fmul_rn(q[c], s);
    }
}

// upd_p / upd_q on the two voxels of a pair in packed form, lane by lane the same
// operations (a lane left inside its ball is scaled by 1, which is exact)
__device__ __forceinline__ void upd_p2(float2 p[3], const float2 g[3], const float2 vb[3], float sigma, float alpha1,
                                       float a1sq)
{
    const float2 s2 = bc2(sigma);
#pragma unroll
    for (int c = 0; c < 3; ++c) p[c] = fma2(s2, sub2(g[c], vb[c]), p[c]);
    const float2 n2 = fma2(p[2], p[2], fma2(p[1], p[1], mul2(p[0], p[0])));
    if (n2.x > a1sq || n2.y > a1sq) {
        const float2 s = make_float2(n2.x > a1sq ? __fmul_rn(alpha1, rsqrtf(n2.x)) : 1.0f,
                                     n2.y > a1sq ? __fmul_rn(alpha1, rsqrtf(n2.y)) : 1.0f);
#pragma unroll
        for (int c = 0; c < 3; ++c) p[c] = mul2(p[c], s);
    }
}

__device__ __forceinline__ void upd_q2(float2 q[6], const float2 dm[3][3], float sigma, float alpha0, float a0sq)
{
    const float2 s2 = bc2(sigma), h2 = bc2(0.5f);
    q[0] = fma2(s2, dm[0][0], q[0]);
    q[1] = fma2(s2, dm[1][1], q[1]);
    q[2] = fma2(s2, dm[2][2], q[2]);
    q[3] = fma2(s2, mul2(h2, add2(dm[0][1], dm[1][0])), q[3]);
    q[4] = fma2(s2, mul2(h2, add2(dm[0][2], dm[2][0])), q[4]);
    q[5] = fma2(s2, mul2(h2, add2(dm[1][2], dm[2][1])), q[5]);
    const float2 off = fma2(q[5], q[5], fma2(q[4], q[4], mul2(q[3], q[3])));
    const float2 n2 = fma2(bc2(2.0f), off, fma2(q[2], q[2], fma2(q[1], q[1], mul2(q[0], q[0]))));
    if (n2.x > a0sq || n2.y > a0sq) {
        const float2 s = make_float2(n2.x > a0sq ? __fmul_rn(alpha0, rsqrtf(n2.x)) : 1.0f,
                                     n2.y > a0sq ? __fmul_rn(alpha0, rsqrtf(n2.y)) : 1.0f);
#pragma unroll
        for (int c = 0; c < 6; ++c) q[c] = mul2(q[c], s);
    }
}

// v <- v + tau (p + div2 q) and its over-relaxation 2 v_new - v_old
__device__ __forceinline__ float vnew(float v0, float p, float d2, float tau)
{
    return __fmaf_rn(tau, __fadd_rn(p, d2), v0);
}
__device__ __forceinline__ float vbar_of(float v1, float v0) { return __fsub_rn(__fmul_rn(2.0f, v1), v0); }

// new p for the halo pair (2hj, 7, hw) / (2hj, hw, 7) on the -AX face (AX = 1: y, 2: z),
// rounded as the owner stores it (D, scales dsc / isc)
template <typename D, int AX, bool KU>
__device__ __forceinline__ void halo_p_pair(const float* h, uint32_t hm, const float* sub, float* hal_p, int tk,
                                            float sigma, float alpha1, float a1sq, float dsc, float isc)
{
    constexpr int OA = 3 - AX;  // the other face axis
    const int hj = tk & 3, hw = tk >> 2;
    const uint32_t lo = AX == 1 ? 2 * hj + 64 * hw : 2 * hj + 8 * hw;  // own voxel at coordinate 0 along AX
    const float2 own = ldf2(sub + lo);
    const float2 u01 = make_float2(h[0], h[1]);
    float2 g[3];
    g[0] = sub2(make_float2(h[1], h[2]), u01);  // x-forward of voxel 0 is voxel 1
    if (!(hm & 1u)) g[0].y = 0.0f;
    g[AX] = sub2(own, u01);
    g[OA] = (hm & 2u) ? sub2(make_float2(h[4], h[5]), u01) : zero2();
    float2 pp[3] = {make_float2(h[12], h[13]), make_float2(h[14], h[15]), make_float2(h[16], h[17])};
    const float2 vv[3] = {make_float2(h[6], h[7]), make_float2(h[8], h[9]), make_float2(h[10], h[11])};
    upd_p2(pp, g, vv, sigma, alpha1, a1sq);
    const int fi = 2 * hj + 8 * hw;
#pragma unroll
    for (int c = 0; c < 3; ++c)
        stf2(hal_p + c * 192 + AX * 64 + fi, KU ? fxk_round2(pp[c]) : DRound2<D>::r(pp[c], dsc, isc));
}

// new q for the halo pair (2hj, 0, hw) / (2hj, hw, 0) on the +AX face, rounded as stored
template <typename S, typename D, int AX, bool KU>
__device__ __forceinline__ void halo_q_pair(const float* h, uint32_t hm, const S* svb, float* hal_q, int tk,
                                            float sigma, float alpha0, float a0sq, float dsc, float isc)
{
    constexpr int OA = 3 - AX;
    const int hj = tk & 3, hw = tk >> 2;
    const uint32_t lo = AX == 1 ? 2 * hj + 56 + 64 * hw : 2 * hj + 8 * hw + 448;  // own voxel at coordinate 7
    float2 dm[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float2 own = Pair<S>::ld(svb + c * 512 + lo);
        const float2 v2 = make_float2(h[2 * c], h[2 * c + 1]);
        dm[0][c] = sub2(v2, make_float2(h[6 + 2 * c], h[2 * c]));  // backward x of voxel 1 is voxel 0
        if (!(hm & 1u)) dm[0][c].x = 0.0f;
        dm[AX][c] = sub2(v2, own);
        dm[OA][c] = (hm & 2u) ? sub2(v2, make_float2(h[12 + 2 * c], h[13 + 2 * c])) : zero2();
    }
    float2 e[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) e[c] = make_float2(h[18 + 2 * c], h[19 + 2 * c]);
    upd_q2(e, dm, sigma, alpha0, a0sq);
    const int fi = 2 * hj + 8 * hw;
#pragma unroll
    for (int c = 0; c < 6; ++c)
        stf2(hal_q + c * 192 + AX * 64 + fi, KU ? fxk_round2(e[c]) : DRound2<D>::r(e[c], dsc, isc));
}

}  // namespace

// Shared-memory layout of a paired CTA: two stages (one brick's u, ubar, v, vbar, p, q
// and packed histogram each; a brick's new duals replace its old ones in place), the halo
// duals of each stage, two neighbour rows, three mbarriers.
struct PairLayout {
    uint32_t tx, stage, pn_bytes, off_pn, off_hal, off_nbr, off_bar, end;
};
__host__ __device__ constexpr PairLayout pair_layout(uint32_t sb, uint32_t sd, uint32_t npairs)
{
    PairLayout L{};
    L.tx = 4096 + (6 * sb + 9 * sd) * 512 + npairs * 2048;
    L.stage = (L.tx + 127) / 128 * 128;
    L.pn_bytes = 0;  // new duals live in the stage (16-bit ones rounded as stored)
    L.off_pn = 2 * L.stage;
    L.off_hal = L.off_pn + 2 * L.pn_bytes;
    L.off_nbr = L.off_hal + 2 * 9 * 192 * 4;
    L.off_bar = (L.off_nbr + 2 * TGV_NNBR * 4 + 15) / 16 * 16;
    L.end = L.off_bar + 3 * 8;
    return L;
}

template <typename S, typename D>
struct PairArgs {
    IterArgs<S, D> it;
    int* err;
    long long wait_budget;             // cycles per wait for a stage (tgv_params.wait_cycles)
    int wait_test;                     // 1: the prologue waits on a barrier nothing completes
    uint32_t stage_bytes, tx_bytes;
    uint32_t pn_bytes;                 // bytes of one own-new-dual buffer (0 when it aliases the stage)
    uint32_t off_pn, off_hal, off_nbr, off_bar;
    uint32_t xrun;                     // work items per run (>= 1)
};

// Per-thread view of one CTA: thread t < 256 owns the voxel pair (2j, y, z), (2j+1, y, z).
//
// Halo tasks (warp-uniform).  Without HW thread t takes item k = t - (first t of its
// range) of the task whose range of the table below holds t.  With HW threads 0-255 take
// none; halo warps 8, 9, 10, 11 take the -y p, -z p, +y q and +z q pair task (item = lane)
// and then, unless that x face is handed over, items 32 * (warp & 1) + lane of the -x p
// task (warps 8, 9) or of the +x q task (warps 10, 11):
//   [0,64)    new p, -x face, single voxel (7, y, z) of the -x brick, y = k&7, z = k>>3
//   [64,96)   new p, -y face, pair (2j, 7, z), (2j+1, 7, z), j = k&3, z = k>>2
//   [96,128)  new p, -z face, pair (2j, y, 7), (2j+1, y, 7), j = k&3, y = k>>2
//   [128,192) new q, +x face, single voxel (0, y, z) of the +x brick
//   [192,224) new q, +y face, pair (2j, 0, z), (2j+1, 0, z)
//   [224,256) new q, +z face, pair (2j, y, 0), (2j+1, y, 0)
// Halo arrays of a stage: hal_p[c][a*64 + face index] (3 x 192 floats), then
// hal_q[c][a*64 + face index] (6 x 192); face index y+8z (a = x), x+8z (a = y), x+8y (a = z).
// Within a run ("hand-over" from brick i to the adjacent item i+1, its +x neighbour):
//   * task 0 of brick i+1 is skipped: phase A of brick i writes hal_p[0][y+8z] of
//     brick i+1's stage from its own new p;
//   * task 3 of brick i is skipped: phase B of brick i parks the partial div2 q sum of
//     its x = 7 voxels in hal_q[qidx(0,c)][y+8z] of its own stage (the slots task 3
//     would have filled); phase A of brick i+1 adds its new q and stores v, vbar.
template <typename S, typename D, int NB, bool HW = false>
struct PairCta {
    using PS = Pair<S>;
    using DP = DPair<D>;
    static constexpr uint32_t SB = sizeof(S), SD = sizeof(D);
    static constexpr uint32_t O_U = 0, O_UB = 2048, O_V = 4096, O_VB = O_V + 3 * 512 * SB,
                              O_P = O_VB + 3 * 512 * SB, O_Q = O_P + 3 * 512 * SD, O_H = O_Q + 6 * 512 * SD;
    static constexpr int NP_MAX = NB ? (NB + 1) / 2 : TGV_MAX_BINS / 2;
    static constexpr int NB_MAX = NB ? NB : TGV_MAX_BINS;
    // with a compile-time bin count every offset is a constant (the launcher uses the same
    // pair_layout); NB = 0 reads them from the arguments
    static constexpr PairLayout LC = pair_layout(SB, SD, NB ? (NB + 1) / 2 : 1);
    // Where the 256-thread form loads the next item's phase A inputs (own boundary values and
    // halo-task inputs): FP32 duals (the batched kernel, two CTAs per SM) into registers
    // before phase B of the current item, so their latency overlaps it; 16-bit duals (three
    // CTAs per SM, 80 registers) just before phase A, the other CTAs' warps covering the
    // latency.  The halo-warp form (HW) has its own placement: own boundary values inside
    // phase B after the prox, face-task inputs by the halo warps at the top of the interval.
    static constexpr bool kEarlyLoads = SD == 4;
    // FX16: every dual of the iteration in units of its fixed-point step (the stored
    // integer), so loads need no product, rounding none either, and the divergences of
    // phase B are exact integer sums scaled once by tau x step
    static constexpr bool kFx = std::is_same<D, int16_t>::value;
    // HW: 384 threads; threads 0-255 own the voxel pairs and do no halo task, and the four
    // halo warps 8-11 compute the halo duals (warp 8 + k takes face task 1, 2, 4, 5 for
    // k = 0..3 and, when that face is not handed over, half of face task 0 (k = 0, 1) or
    // 3 (k = 2, 3)), so the own warps' interval carries no halo work and fewer registers
    static constexpr bool kHW = HW;
    static constexpr int kCtaThreads = HW ? 384 : 256;

    const PairArgs<S, D>& P;
    const IterArgs<S, D>& A;
    unsigned char* smem;
    int t, j, y, z, x0, task, tk, nbk, nbins, npairs;
    bool own;       // this thread owns a voxel pair (all threads unless HW)
    int task2, tk2; // HW halo warps: the x-face task taken when that face is not handed over
    uint32_t l0;
    float sigma, alpha1, alpha0, a1sq, a0sq;  // dual step, projection radii (kFx: 32767 steps)
    float sigp, sigq, taup, tauq;             // kFx: sigma / step and tau x step for p and q

    // inputs of the next brick's phase A held in registers
    float ubf_x;
    float2 ubf_y, ubf_z;
    float vbb_x[3];
    float2 vbb_y[3], vbb_z[3];
    float h[30];
    uint32_t hm;
    int hn;

    // flip: the in and out ping-pong copies of A trade places (the batched kernel's odd
    // iterations of a chunk); false in the level kernel, where the selects fold away
    bool flip;

    __device__ __forceinline__ PairCta(const PairArgs<S, D>& p, unsigned char* sm, bool fl = false)
        : P(p), A(p.it), smem(sm), flip(fl)
    {
        t = threadIdx.x;
        j = t & 3;
        y = (t >> 2) & 7;
        z = t >> 5;
        x0 = 2 * j;
        l0 = x0 + 8 * y + 64 * z;
        if (HW) {
            own = t < 256;
            const int hw = (t >> 5) - 8, lane = t & 31;
            task = own ? -1 : (hw == 0 ? 1 : (hw == 1 ? 2 : (hw == 2 ? 4 : 5)));
            tk = lane;
            task2 = hw < 2 ? 0 : 3;
            tk2 = 32 * (hw & 1) + lane;
        } else {
            own = true;
            task = t < 64 ? 0 : (t < 96 ? 1 : (t < 128 ? 2 : (t < 192 ? 3 : (t < 224 ? 4 : 5))));
            tk = t < 64 ? t : (t < 96 ? t - 64 : (t < 128 ? t - 96 : (t < 192 ? t - 128 : (t < 224 ? t - 192 : t - 224))));
            task2 = tk2 = -1;
        }
        nbk = (int)A.nb;
        nbins = NB ? NB : A.nbins;
        npairs = NB ? (NB + 1) / 2 : A.npairs;
        sigma = A.sigma;
        if constexpr (kFx) {
            sigp = __fmul_rn(A.sigma, A.ds.isp);
            sigq = __fmul_rn(A.sigma, A.ds.isq);
            alpha1 = alpha0 = 32767.0f;
            taup = __fmul_rn(A.tau, A.ds.dsp);
            tauq = __fmul_rn(A.tau, A.ds.dsq);
        } else {
            alpha1 = A.alpha1;
            alpha0 = A.alpha0;
        }
        a1sq = alpha1 * alpha1;
        a0sq = alpha0 * alpha0;
    }

    // step sizes as the iteration applies them (one sigma and tau unless kFx)
    __device__ __forceinline__ float sp_() const { return kFx ? sigp : sigma; }
    __device__ __forceinline__ float sq_() const { return kFx ? sigq : sigma; }
    __device__ __forceinline__ float tp_() const { return kFx ? taup : A.tau; }
    __device__ __forceinline__ float tq_() const { return kFx ? tauq : A.tau; }

    __device__ __forceinline__ const float* ubi() const { return flip ? A.ubar_out : A.ubar_in; }
    __device__ __forceinline__ float* ubo() const { return flip ? const_cast<float*>(A.ubar_in) : A.ubar_out; }
    __device__ __forceinline__ const S* vbi() const { return flip ? A.vbar_out : A.vbar_in; }
    __device__ __forceinline__ S* vbo() const { return flip ? const_cast<S*>(A.vbar_in) : A.vbar_out; }
    __device__ __forceinline__ const D* pin() const { return flip ? A.p_out : A.p_in; }
    __device__ __forceinline__ D* pout() const { return flip ? const_cast<D*>(A.p_in) : A.p_out; }
    __device__ __forceinline__ const D* qin() const { return flip ? A.q_out : A.q_in; }
    __device__ __forceinline__ D* qout() const { return flip ? const_cast<D*>(A.q_in) : A.q_out; }

    __device__ __forceinline__ uint32_t stage_bytes() const { return NB ? LC.stage : P.stage_bytes; }
    __device__ __forceinline__ uint32_t off_pn() const { return NB ? LC.off_pn : P.off_pn; }
    __device__ __forceinline__ uint32_t off_hal() const { return NB ? LC.off_hal : P.off_hal; }
    __device__ __forceinline__ uint32_t off_nbr() const { return NB ? LC.off_nbr : P.off_nbr; }
    __device__ __forceinline__ uint32_t off_bar() const { return NB ? LC.off_bar : P.off_bar; }
    __device__ __forceinline__ uint32_t tx_bytes() const { return NB ? LC.tx : P.tx_bytes; }
    __device__ __forceinline__ unsigned char* stage(int s) const { return smem + (size_t)s * stage_bytes(); }
    // a brick's own new duals, in its stage in place of the old ones (storage type D; FP32
    // or the rounded 16-bit value): pairs and single values at voxel index i of component c
    __device__ __forceinline__ const D* np_(int s) const { return (const D*)(stage(s) + O_P); }
    __device__ __forceinline__ const D* nq_(int s) const { return (const D*)(stage(s) + O_Q); }
    // a dual pair / single value as the iteration handles it (kFx: in step units)
    __device__ __forceinline__ float2 dl2(const D* p, float dsc) const
    {
        if constexpr (kFx) return fxk_ld2((const int16_t*)p);
        else return DP::ld(p, dsc);
    }
    __device__ __forceinline__ float dl1(const D* p, float dsc) const
    {
        if constexpr (kFx) return (float)*(const int16_t*)p;
        else return ld_d(p, dsc);
    }
    __device__ __forceinline__ float2 ldp2(int s, int i) const { return dl2(np_(s) + i, A.ds.dsp); }
    __device__ __forceinline__ float2 ldq2(int s, int i) const { return dl2(nq_(s) + i, A.ds.dsq); }
    __device__ __forceinline__ float ldp1(int s, int i) const { return dl1(np_(s) + i, A.ds.dsp); }
    __device__ __forceinline__ float ldq1(int s, int i) const { return dl1(nq_(s) + i, A.ds.dsq); }
    // stores a new dual pair (rounded to the storage type) and returns the stored values
    __device__ __forceinline__ float2 stp2(int s, int i, float2 v) const
    {
        if constexpr (kFx) return fxk_store2((int16_t*)np_(s) + i, v);
        DRoundStore<D>::st((D*)np_(s) + i, v, A.ds.dsp, A.ds.isp);
        return v;
    }
    __device__ __forceinline__ float2 stq2(int s, int i, float2 v) const
    {
        if constexpr (kFx) return fxk_store2((int16_t*)nq_(s) + i, v);
        DRoundStore<D>::st((D*)nq_(s) + i, v, A.ds.dsq, A.ds.isq);
        return v;
    }
    __device__ __forceinline__ float rp(float x) const
    {
        if constexpr (kFx) return fxk_round(x);
        else return DRound<D>::r(x, A.ds.dsp, A.ds.isp);
    }
    __device__ __forceinline__ float rq(float x) const
    {
        if constexpr (kFx) return fxk_round(x);
        else return DRound<D>::r(x, A.ds.dsq, A.ds.isq);
    }
    // global store of a new dual pair held in the stage: the stored word itself (16-bit), or
    // the FP32 values
    __device__ __forceinline__ void out_p2(int s, int i, D* dst, float2 v) const
    {
        if constexpr (SD == 4) stf2((float*)dst, v);
        else *(uint32_t*)dst = *(const uint32_t*)(np_(s) + i);
    }
    __device__ __forceinline__ void out_q2(int s, int i, D* dst, float2 v) const
    {
        if constexpr (SD == 4) stf2((float*)dst, v);
        else *(uint32_t*)dst = *(const uint32_t*)(nq_(s) + i);
    }
    __device__ __forceinline__ float* hal_p(int s) const { return (float*)(smem + off_hal()) + s * (9 * 192); }
    __device__ __forceinline__ float* hal_q(int s) const { return hal_p(s) + 3 * 192; }
    __device__ __forceinline__ uint64_t* bar() const { return (uint64_t*)(smem + off_bar()); }
    __device__ __forceinline__ int* nbr_row(int s) const { return (int*)(smem + off_nbr()) + s * TGV_NNBR; }

    __device__ __forceinline__ void issue(int s, uint32_t brick) const
    {
        unsigned char* st = stage(s);
        uint64_t* b = bar() + s;
        mbar_arrive_expect_tx(b, tx_bytes());
        bulk_copy_g2s(st + O_U, A.u + (size_t)brick * TGV_BVOX, 2048, b);
        bulk_copy_g2s(st + O_UB, ubi() + (size_t)brick * TGV_BVOX, 2048, b);
        bulk_copy_g2s(st + O_V, A.v + (size_t)brick * 3 * TGV_BVOX, 3 * 512 * SB, b);
        bulk_copy_g2s(st + O_VB, vbi() + (size_t)brick * 3 * TGV_BVOX, 3 * 512 * SB, b);
        bulk_copy_g2s(st + O_P, pin() + (size_t)brick * 3 * TGV_BVOX, 3 * 512 * SD, b);
        bulk_copy_g2s(st + O_Q, qin() + (size_t)brick * 6 * TGV_BVOX, 6 * 512 * SD, b);
        bulk_copy_g2s(st + O_H, A.hist + brick * (size_t)npairs * TGV_BVOX, (uint32_t)npairs * 2048u, b);
    }

    // ---- global loads a brick's phase A needs besides its stage (own boundary neighbours, halo inputs)
    // skip0 / skip3: the -x p halo comes from the previous item, the +x q halo is
    // replaced by the hand-over to the next item (see above)
    __device__ __forceinline__ void load_inputs(const int* nrow, bool skip0, bool skip3)
    {
        load_own(nrow);
        load_halo(nrow, task, tk, skip0, skip3);
    }

    // the own pair's boundary neighbours in adjacent bricks
    __device__ __forceinline__ void load_own(const int* nrow)
    {
        const int n_px = nrow[NB_PX], n_mx = nrow[NB_MX], n_py = nrow[NB_PY], n_my = nrow[NB_MY];
        const int n_pz = nrow[NB_PZ], n_mz = nrow[NB_MZ];
        ubf_x = 0.0f;
        ubf_y = ubf_z = make_float2(0, 0);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            vbb_x[c] = 0.0f;
            vbb_y[c] = vbb_z[c] = make_float2(0, 0);
        }
        if (j == 3 && n_px >= 0) ubf_x = ubi()[(size_t)n_px * TGV_BVOX + l0 + 1 - 7];
        if (y == 7 && n_py >= 0) ubf_y = ldf2(ubi() + (size_t)n_py * TGV_BVOX + l0 - 56);
        if (z == 7 && n_pz >= 0) ubf_z = ldf2(ubi() + (size_t)n_pz * TGV_BVOX + l0 - 448);
        if (j == 0 && n_mx >= 0) {
#pragma unroll
            for (int c = 0; c < 3; ++c) vbb_x[c] = ld_s(vbi() + ((size_t)n_mx * 3 + c) * TGV_BVOX + l0 + 7);
        }
        if (y == 0 && n_my >= 0) {
#pragma unroll
            for (int c = 0; c < 3; ++c) vbb_y[c] = PS::ld(vbi() + ((size_t)n_my * 3 + c) * TGV_BVOX + l0 + 56);
        }
        if (z == 0 && n_mz >= 0) {
#pragma unroll
            for (int c = 0; c < 3; ++c) vbb_z[c] = PS::ld(vbi() + ((size_t)n_mz * 3 + c) * TGV_BVOX + l0 + 448);
        }
    }

    // halo inputs of face task `task`, item tk (task < 0: none).  p tasks: h[0..1]
    // ubar(h0,h1), h[2..3] forward along the first face axis, h[4..5] along the second,
    // h[6..11] vbar (3 x pair), h[12..17] p (3 x pair).  q tasks: h[0..5] vbar (3 x pair),
    // h[6..11] backward along the first face axis, h[12..17] along the second, h[18..29] q
    // (6 x pair).  Singles use the even slots.
    __device__ __forceinline__ void load_halo(const int* nrow, int task, int tk, bool skip0, bool skip3)
    {
        hm = 0;
        hn = -1;
        if (HW && task < 0) return;
        {
            const int a = task % 3;
            hn = task < 3 ? nrow[nb_minus(a)] : nrow[nb_plus(a)];
            if (hn >= nbk) hn = -1;  // frozen: no dual variables there
            if ((task == 0 && skip0) || (task == 3 && skip3)) hn = -1;
        }
        if (hn < 0) return;
        // the halo brick's fields: base pointers once, constant offsets per load
        const float* ubn = ubi() + (size_t)hn * TGV_BVOX;
        const S* vbn = vbi() + (size_t)hn * 3 * TGV_BVOX;
        const D* pnb = pin() + (size_t)hn * 3 * TGV_BVOX;
        const D* qnb = qin() + (size_t)hn * 6 * TGV_BVOX;
        if (task == 0) {  // -x face single: (7, hy, hz)
            const int hy = tk & 7, hz = tk >> 3;
            const uint32_t lh = 7 + 8 * hy + 64 * hz;
            h[0] = ubn[lh];
            if (hy < 7) {
                h[2] = ubn[lh + 8];
                hm |= 1u;
            } else if (nrow[NB_MX_PY] >= 0) {
                h[2] = ubi()[(size_t)nrow[NB_MX_PY] * TGV_BVOX + lh - 56];
                hm |= 1u;
            }
            if (hz < 7) {
                h[4] = ubn[lh + 64];
                hm |= 2u;
            } else if (nrow[NB_MX_PZ] >= 0) {
                h[4] = ubi()[(size_t)nrow[NB_MX_PZ] * TGV_BVOX + lh - 448];
                hm |= 2u;
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                h[6 + 2 * c] = ld_s(vbn + c * TGV_BVOX + lh);
                h[12 + 2 * c] = dl1(pnb + c * TGV_BVOX + lh, A.ds.dsp);
            }
        } else if (task == 1 || task == 2) {  // -y / -z face pairs
            const int hj = tk & 3, hw = tk >> 2;  // hw = z (task 1) or y (task 2)
            const uint32_t lh = task == 1 ? 2 * hj + 56 + 64 * hw : 2 * hj + 8 * hw + 448;
            float2 u2 = ldf2(ubn + lh);
            h[0] = u2.x;
            h[1] = u2.y;
            if (hj < 3) {  // forward along x of the pair's second voxel
                h[2] = ubn[lh + 2];
                hm |= 1u;
            } else {
                const int e = nrow[task == 1 ? NB_MY_PX : NB_MZ_PX];
                if (e >= 0) {
                    h[2] = ubi()[(size_t)e * TGV_BVOX + lh + 1 - 7];
                    hm |= 1u;
                }
            }
            const uint32_t ostr = task == 1 ? 64 : 8;  // the other face axis: z (task 1) or y (task 2)
            if (hw < 7) {
                u2 = ldf2(ubn + lh + ostr);
                h[4] = u2.x;
                h[5] = u2.y;
                hm |= 2u;
            } else {
                const int e = nrow[task == 1 ? NB_MY_PZ : NB_MZ_PY];
                if (e >= 0) {
                    u2 = ldf2(ubi() + (size_t)e * TGV_BVOX + lh - 7 * ostr);
                    h[4] = u2.x;
                    h[5] = u2.y;
                    hm |= 2u;
                }
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float2 w = PS::ld(vbn + c * TGV_BVOX + lh);
                h[6 + 2 * c] = w.x;
                h[7 + 2 * c] = w.y;
                w = dl2(pnb + c * TGV_BVOX + lh, A.ds.dsp);
                h[12 + 2 * c] = w.x;
                h[13 + 2 * c] = w.y;
            }
        } else if (task == 3) {  // +x face single: (0, hy, hz)
            const int hy = tk & 7, hz = tk >> 3;
            const uint32_t lh = 8 * hy + 64 * hz;
#pragma unroll
            for (int c = 0; c < 3; ++c) h[2 * c] = ld_s(vbn + c * TGV_BVOX + lh);
            if (hy > 0) {
#pragma unroll
                for (int c = 0; c < 3; ++c) h[6 + 2 * c] = ld_s(vbn + c * TGV_BVOX + lh - 8);
                hm |= 1u;
            } else if (nrow[NB_MY_PX] >= 0) {
                const size_t e = (size_t)nrow[NB_MY_PX];
#pragma unroll
                for (int c = 0; c < 3; ++c) h[6 + 2 * c] = ld_s(vbi() + (e * 3 + c) * TGV_BVOX + lh + 56);
                hm |= 1u;
            }
            if (hz > 0) {
#pragma unroll
                for (int c = 0; c < 3; ++c) h[12 + 2 * c] = ld_s(vbn + c * TGV_BVOX + lh - 64);
                hm |= 2u;
            } else if (nrow[NB_MZ_PX] >= 0) {
                const size_t e = (size_t)nrow[NB_MZ_PX];
#pragma unroll
                for (int c = 0; c < 3; ++c) h[12 + 2 * c] = ld_s(vbi() + (e * 3 + c) * TGV_BVOX + lh + 448);
                hm |= 2u;
            }
#pragma unroll
            for (int c = 0; c < 6; ++c) h[18 + 2 * c] = dl1(qnb + c * TGV_BVOX + lh, A.ds.dsq);
        } else {  // task 4 / 5: +y / +z face pairs
            const int hj = tk & 3, hw = tk >> 2;  // hw = z (task 4) or y (task 5)
            const uint32_t lh = task == 4 ? 2 * hj + 64 * hw : 2 * hj + 8 * hw;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float2 w = PS::ld(vbn + c * TGV_BVOX + lh);
                h[2 * c] = w.x;
                h[2 * c + 1] = w.y;
            }
            if (hj > 0) {  // backward along x of the pair's first voxel
#pragma unroll
                for (int c = 0; c < 3; ++c) h[6 + 2 * c] = ld_s(vbn + c * TGV_BVOX + lh - 1);
                hm |= 1u;
            } else {
                const int e = nrow[task == 4 ? NB_MX_PY : NB_MX_PZ];
                if (e >= 0) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) h[6 + 2 * c] = ld_s(vbi() + ((size_t)e * 3 + c) * TGV_BVOX + lh + 7);
                    hm |= 1u;
                }
            }
            const uint32_t ostr = task == 4 ? 64 : 8;  // the other face axis: z (task 4) or y (task 5)
            if (hw > 0) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float2 w = PS::ld(vbn + c * TGV_BVOX + lh - ostr);
                    h[12 + 2 * c] = w.x;
                    h[13 + 2 * c] = w.y;
                }
                hm |= 2u;
            } else {
                const int e = nrow[task == 4 ? NB_MZ_PY : NB_MY_PZ];
                if (e >= 0) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float2 w = PS::ld(vbi() + ((size_t)e * 3 + c) * TGV_BVOX + lh + 7 * ostr);
                        h[12 + 2 * c] = w.x;
                        h[13 + 2 * c] = w.y;
                    }
                    hm |= 2u;
                }
            }
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                const float2 w = dl2(qnb + c * TGV_BVOX + lh, A.ds.dsq);
                h[18 + 2 * c] = w.x;
                h[19 + 2 * c] = w.y;
            }
        }
    }

    // ---- phase A of the brick in stage s: new p, q at the own pair (into the stage, in
    // place of the old ones) and the halo duals (into hal_p / hal_q).  Returns the link bits phase B needs.
    // from_prev: this brick is the +x neighbour and run successor of brick bprev, whose
    // phase B parked the partial v update of its x = 7 voxels (completed here);
    // to_next: the next item is this brick's +x neighbour (its -x halo p is written here).
    __device__ __forceinline__ uint32_t phase_a(int s, const int* nrow, bool from_prev, bool to_next, uint32_t bprev)
    {
        own_update(s, nrow, from_prev, to_next, bprev);
        halo_compute(s, task, tk);
        return link_bits(nrow);
    }

    // HW halo warps: the face task whose inputs are in h, then the x-face task unless
    // that face is handed over (its inputs loaded here, after the first task)
    __device__ __forceinline__ void halo_phase(int s, const int* nrow, bool skip0, bool skip3)
    {
        halo_compute(s, task, tk);
        load_halo(nrow, task2, tk2, skip0, skip3);
        halo_compute(s, task2, tk2);
    }

    // the own pair's part of phase A; returns the link bits phase B needs
    __device__ __forceinline__ uint32_t phase_a_own(int s, const int* nrow, bool from_prev, bool to_next,
                                                    uint32_t bprev)
    {
        own_update(s, nrow, from_prev, to_next, bprev);
        return link_bits(nrow);
    }

    __device__ __forceinline__ void own_update(int s, const int* nrow, bool from_prev, bool to_next, uint32_t bprev)
    {
        const int n_px = nrow[NB_PX], n_mx = nrow[NB_MX], n_py = nrow[NB_PY], n_my = nrow[NB_MY];
        const int n_pz = nrow[NB_PZ], n_mz = nrow[NB_MZ];
        unsigned char* st = stage(s);
        const float* sub = (const float*)(st + O_UB);
        const S* svb = (const S*)(st + O_VB);
        const D* sp = (const D*)(st + O_P);
        const D* sq = (const D*)(st + O_Q);
        const float2 ub = ldf2(sub + l0);
        float2 vb[3], pn[3], qn[6];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            vb[c] = PS::ld(svb + c * 512 + l0);
            pn[c] = dl2(sp + c * 512 + l0, A.ds.dsp);
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) qn[c] = dl2(sq + c * 512 + l0, A.ds.dsq);
        const bool fx1 = j < 3 || n_px >= 0, fy = y < 7 || n_py >= 0, fz = z < 7 || n_pz >= 0;
        const bool bx0 = j > 0 || n_mx >= 0, by = y > 0 || n_my >= 0, bz = z > 0 || n_mz >= 0;
        {
            const float2 uy = y < 7 ? ldf2(sub + l0 + 8) : ubf_y;
            const float2 uz = z < 7 ? ldf2(sub + l0 + 64) : ubf_z;
            const float ux1 = j < 3 ? sub[l0 + 2] : ubf_x;
            float2 g[3];
            g[0] = sub2(make_float2(ub.y, ux1), ub);  // x-forward: voxel 1 of voxel 0, x0 + 2 of voxel 1
            if (!fx1) g[0].y = 0.0f;
            g[1] = fy ? sub2(uy, ub) : zero2();
            g[2] = fz ? sub2(uz, ub) : zero2();
            float2 dm[3][3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float wx0 = j > 0 ? ld_s(svb + c * 512 + l0 - 1) : vbb_x[c];
                const float2 wy = y > 0 ? PS::ld(svb + c * 512 + l0 - 8) : vbb_y[c];
                const float2 wz = z > 0 ? PS::ld(svb + c * 512 + l0 - 64) : vbb_z[c];
                dm[0][c] = sub2(vb[c], make_float2(wx0, vb[c].x));  // x-backward: x0 - 1 of voxel 0, voxel 0 of voxel 1
                if (!bx0) dm[0][c].x = 0.0f;
                dm[1][c] = by ? sub2(vb[c], wy) : zero2();
                dm[2][c] = bz ? sub2(vb[c], wz) : zero2();
            }
            upd_p2(pn, g, vb, sp_(), alpha1, a1sq);
            upd_q2(qn, dm, sq_(), alpha0, a0sq);
        }
        // the values the level stores (16-bit duals rounded once); own old p / q were read
        // above by this thread only: overwrite them in place
#pragma unroll
        for (int c = 0; c < 3; ++c) pn[c] = stp2(s, c * 512 + l0, pn[c]);
#pragma unroll
        for (int c = 0; c < 6; ++c) qn[c] = stq2(s, c * 512 + l0, qn[c]);
        // hand-over along the run
        if (to_next && j == 3) hal_p(s ^ 1)[y + 8 * z] = pn[0].y;
        if (from_prev && j == 0) {
            // brick bprev's voxel (7, y, z): its partial div2 q, its new p and old v are
            // still in the other stage; add the x-forward term (this voxel's new q)
            const int ps = s ^ 1;
            const float* hq_prev = hal_q(ps);
            const S* sv_prev = (const S*)(stage(ps) + O_V);
            const S* svb_prev = (const S*)(stage(ps) + O_VB);
            const uint32_t l6 = 6 + 8 * y + 64 * z;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int qc = qidx(0, c);
                // (16-bit duals: the stored value read back from the stage, decoded as phase B
                // decodes it, rather than the register copy of the packed rounding)
                const float qx0 = SD == 4 ? qn[qc].x : ldq1(s, qc * 512 + l0);
                const float d2 = __fadd_rn(hq_prev[qc * 192 + y + 8 * z], qx0);
                const float v0 = ld_s(sv_prev + c * 512 + l6 + 1);
                const float p7 = ldp1(ps, c * 512 + l6 + 1);
                const float v1 = kFx ? __fmaf_rn(tp_(), p7, __fmaf_rn(tq_(), d2, v0)) : vnew(v0, p7, d2, A.tau);
                // with the x = 6 values parked by its phase B: one pair store per field
                const size_t oi = ((size_t)bprev * 3 + c) * TGV_BVOX + l6;
                PS::st(A.v + oi, make_float2(ld_s(sv_prev + c * 512 + l6), v1));
                PS::st(vbo() + oi, make_float2(ld_s(svb_prev + c * 512 + l6), vbar_of(v1, v0)));
            }
        }

    }

    // link bits for phase B: bit 2k "any", bit 2k+1 "active", k = 0 (-x of voxel 0),
    // 1 (+x of voxel 1), 2 (+y), 3 (-y), 4 (+z), 5 (-z)
    __device__ __forceinline__ uint32_t link_bits(const int* nrow) const
    {
        const int n_px = nrow[NB_PX], n_mx = nrow[NB_MX], n_py = nrow[NB_PY], n_my = nrow[NB_MY];
        const int n_pz = nrow[NB_PZ], n_mz = nrow[NB_MZ];
        const bool fx1 = j < 3 || n_px >= 0, fy = y < 7 || n_py >= 0, fz = z < 7 || n_pz >= 0;
        const bool bx0 = j > 0 || n_mx >= 0, by = y > 0 || n_my >= 0, bz = z > 0 || n_mz >= 0;
        uint32_t L = 0;
        L |= (bx0 ? 1u : 0u) | ((j > 0 || (n_mx >= 0 && n_mx < nbk)) ? 2u : 0u);
        L |= (fx1 ? 4u : 0u) | ((j < 3 || (n_px >= 0 && n_px < nbk)) ? 8u : 0u);
        L |= (fy ? 16u : 0u) | ((y < 7 || (n_py >= 0 && n_py < nbk)) ? 32u : 0u);
        L |= (by ? 64u : 0u) | ((y > 0 || (n_my >= 0 && n_my < nbk)) ? 128u : 0u);
        L |= (fz ? 256u : 0u) | ((z < 7 || (n_pz >= 0 && n_pz < nbk)) ? 512u : 0u);
        L |= (bz ? 1024u : 0u) | ((z > 0 || (n_mz >= 0 && n_mz < nbk)) ? 2048u : 0u);
        return L;
    }

    // the halo duals of face task `task`, item tk, from the inputs in h (hn < 0: none)
    __device__ __forceinline__ void halo_compute(int s, int task, int tk)
    {
        unsigned char* st = stage(s);
        const float* sub = (const float*)(st + O_UB);
        const S* svb = (const S*)(st + O_VB);
        float* hp = hal_p(s);
        float* hq = hal_q(s);
        if (hn >= 0) {
            if (task == 0) {  // p at (7, hy, hz) of the -x brick
                const int hy = tk & 7, hz = tk >> 3;
                const float g[3] = {sub[8 * hy + 64 * hz] - h[0], (hm & 1u) ? h[2] - h[0] : 0.0f,
                                    (hm & 2u) ? h[4] - h[0] : 0.0f};
                float pp[3] = {h[12], h[14], h[16]};
                const float vv[3] = {h[6], h[8], h[10]};
                upd_p(pp, g, vv, sp_(), alpha1, a1sq);
#pragma unroll
                for (int c = 0; c < 3; ++c) hp[c * 192 + tk] = rp(pp[c]);
            } else if (task == 1) {
                halo_p_pair<D, 1, kFx>(h, hm, sub, hp, tk, sp_(), alpha1, a1sq, A.ds.dsp, A.ds.isp);
            } else if (task == 2) {
                halo_p_pair<D, 2, kFx>(h, hm, sub, hp, tk, sp_(), alpha1, a1sq, A.ds.dsp, A.ds.isp);
            } else if (task == 3) {  // q at (0, hy, hz) of the +x brick
                const int hy = tk & 7, hz = tk >> 3;
                const uint32_t lo = 7 + 8 * hy + 64 * hz;
                float dm[3][3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    dm[0][c] = h[2 * c] - ld_s(svb + c * 512 + lo);
                    dm[1][c] = (hm & 1u) ? h[2 * c] - h[6 + 2 * c] : 0.0f;
                    dm[2][c] = (hm & 2u) ? h[2 * c] - h[12 + 2 * c] : 0.0f;
                }
                float e[6];
#pragma unroll
                for (int c = 0; c < 6; ++c) e[c] = h[18 + 2 * c];
                upd_q(e, dm, sq_(), alpha0, a0sq);
#pragma unroll
                for (int c = 0; c < 6; ++c) hq[c * 192 + tk] = rq(e[c]);
            } else if (task == 4) {
                halo_q_pair<S, D, 1, kFx>(h, hm, svb, hq, tk, sq_(), alpha0, a0sq, A.ds.dsq, A.ds.isq);
            } else {
                halo_q_pair<S, D, 2, kFx>(h, hm, svb, hq, tk, sq_(), alpha0, a0sq, A.ds.dsq, A.ds.isq);
            }
        }
    }

    // ---- phase B of brick b in stage s: divergences, prox, over-relaxation, global stores.
    // to_next: the next item is b's +x neighbour; the v update of the x = 7 voxels is
    // parked without its x-forward div2 q term and completed by that item's phase A.
    // nrow_next (HW own threads): the next item's neighbour row; its own pairs' boundary
    // inputs (load_own) are loaded right after the prox, where the registers the prox
    // needed are free, so the v update and the stores cover their latency.
    __device__ __forceinline__ void phase_b(int s, uint32_t b, uint32_t L, bool to_next, const int* nrow_next = nullptr)
    {
        unsigned char* st = stage(s);
        const float* su = (const float*)(st + O_U);
        const S* sv = (const S*)(st + O_V);
        const uint32_t* sh = (const uint32_t*)(st + O_H);
        const float* hp = hal_p(s);
        const float* hq = hal_q(s);
        float2 pn[3], qn[6];
#pragma unroll
        for (int c = 0; c < 3; ++c) pn[c] = ldp2(s, c * 512 + l0);
#pragma unroll
        for (int c = 0; c < 6; ++c) qn[c] = ldq2(s, c * 512 + l0);
        // div1 p (d1) and div2 q (d2[c]) of the pair, accumulated term by term
        // x: voxel 0: forward = voxel 1, backward = (x0-1) or the -x brick;
        //    voxel 1: backward = voxel 0, forward = (x0+2) or the +x brick
        // (voxel 1's x-forward div2 q term is added last, after y and z)
        float2 d1 = sub2(make_float2(pn[0].x, (L & 4u) ? pn[0].y : 0.0f),
                         make_float2((L & 2u) ? (j > 0 ? ldp1(s, l0 - 1) : hp[y + 8 * z]) : 0.0f, pn[0].x));
        float2 d2[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int qc = qidx(0, c);
            d2[c] = sub2(make_float2(qn[qc].y, 0.0f), make_float2((L & 1u) ? qn[qc].x : 0.0f, qn[qc].y));
        }
        // y
        const uint32_t fyi = 64 + x0 + 8 * z;
        if (L & 16u) d1 = add2(d1, pn[1]);
        if (L & 128u) d1 = sub2(d1, y > 0 ? ldp2(s, 512 + l0 - 8) : ldf2(hp + 192 + fyi));
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int qc = qidx(1, c);
            if (L & 32u) d2[c] = add2(d2[c], y < 7 ? ldq2(s, qc * 512 + l0 + 8) : ldf2(hq + qc * 192 + fyi));
            if (L & 64u) d2[c] = sub2(d2[c], qn[qc]);
        }
        // z
        const uint32_t fzi = 128 + x0 + 8 * y;
        if (L & 256u) d1 = add2(d1, pn[2]);
        if (L & 2048u) d1 = sub2(d1, z > 0 ? ldp2(s, 1024 + l0 - 64) : ldf2(hp + 384 + fzi));
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int qc = qidx(2, c);
            if (L & 512u) d2[c] = add2(d2[c], z < 7 ? ldq2(s, qc * 512 + l0 + 64) : ldf2(hq + qc * 192 + fzi));
            if (L & 1024u) d2[c] = sub2(d2[c], qn[qc]);
        }
        // the new q are final.  FP32: store them now, so their registers are free for the
        // prox; 16-bit duals store the word held in the stage, at the end
        if constexpr (SD == 4) {
#pragma unroll
            for (int c = 0; c < 6; ++c) out_q2(s, c * 512 + l0, qout() + ((size_t)b * 6 + c) * TGV_BVOX + l0, qn[c]);
        }
        const float2 u0 = ldf2(su + l0);
        const float2 ut = fma2(bc2(tp_()), d1, u0);
        // prox: generalised median = max_i min(ut - tau*lambda*W_i, c_i), c_n = +inf
        // total counts in integers (exact; the same value as a float sum, which is exact
        // below 2^24), one conversion each
        uint32_t hwa[NP_MAX], hwb[NP_MAX];
        uint32_t hsa = 0u, hsb = 0u;
#pragma unroll
        for (int k = 0; k < NP_MAX; ++k) {
            uint2 w = make_uint2(0u, 0u);
            if (NB || k < npairs) w = *(const uint2*)(sh + k * 512 + l0);
            hwa[k] = w.x;
            hwb[k] = w.y;
            hsa += (w.x & 0xffffu) + (w.x >> 16);
            hsb += (w.y & 0xffffu) + (w.y >> 16);
        }
        float2 W = make_float2(-(float)hsa, -(float)hsb);
        const float2 ntl = bc2(-A.taulam);
        float una = -INFINITY, unb = -INFINITY;
#pragma unroll
        for (int i = 0; i < NB_MAX; ++i) {
            if (NB || i < nbins) {
                const float ci = A.c[i];
                const float2 cand = fma2(ntl, W, ut);
                una = fmaxf(una, fminf(cand.x, ci));
                unb = fmaxf(unb, fminf(cand.y, ci));
                // count i as a float without an integer conversion: its 16 bits as the
                // mantissa of 2^23 (a byte permute), minus 2^23 (exact)
                const uint32_t sel = (i & 1) ? 0x7632u : 0x7610u;
                const float2 hf = sub2(make_float2(__uint_as_float(__byte_perm(hwa[i >> 1], 0x4B000000u, sel)),
                                                   __uint_as_float(__byte_perm(hwb[i >> 1], 0x4B000000u, sel))),
                                       bc2(8388608.0f));
                W = fma2(bc2(2.0f), hf, W);
            }
        }
        {
            const float2 cand = fma2(ntl, W, ut);
            una = fmaxf(una, cand.x);
            unb = fmaxf(unb, cand.y);
        }
        if (A.clamp_u) {
            una = fminf(1.0f, fmaxf(-1.0f, una));
            unb = fminf(1.0f, fmaxf(-1.0f, unb));
        }
        const float2 un = make_float2(una, unb);
        if (nrow_next) load_own(nrow_next);
        const size_t vi = (size_t)b * TGV_BVOX + l0;
        stf2(A.u + vi, un);
        stf2(ubo() + vi, sub2(add2(un, un), u0));
        const bool park = to_next && j == 3;  // uniform per warp row group; implies L & 8
        const float2 tau2 = bc2(A.tau);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t oi = ((size_t)b * 3 + c) * TGV_BVOX + l0;
            const float2 v0 = PS::ld(sv + c * 512 + l0);
            // every lane forms the pair (a parking lane's x = 7 value is not used), so
            // only the stores below depend on the lane
            const float part = d2[c].y;
            const float fwdq = j < 3 ? ldq1(s, qidx(0, c) * 512 + l0 + 2) : hq[qidx(0, c) * 192 + y + 8 * z];
            const float2 d2c = make_float2(d2[c].x, (L & 8u) ? __fadd_rn(part, fwdq) : part);
            // v <- v + tau (p + div2 q), vbar = 2 v_new - v_old (vnew / vbar_of lane by lane)
            const float2 v1 =
                kFx ? fma2(bc2(tp_()), pn[c], fma2(bc2(tq_()), d2c, v0)) : fma2(tau2, add2(pn[c], d2c), v0);
            const float2 vb1 = sub2(add2(v1, v1), v0);
            if (park) {
                // x = 6 is final, x = 7 waits for the next item's q: keep both stores as one
                // pair store (no split sectors) by parking x = 6's new v and vbar in this
                // stage's v and vbar slots, which nothing reads any more
                hal_q(s)[qidx(0, c) * 192 + y + 8 * z] = part;
                st_s((S*)(st + O_V) + c * 512 + l0, v1.x);
                st_s((S*)(st + O_VB) + c * 512 + l0, vb1.x);
            } else {
                PS::st(A.v + oi, v1);
                PS::st(vbo() + oi, vb1);
            }
            out_p2(s, c * 512 + l0, pout() + oi, pn[c]);
        }
        if constexpr (SD != 4) {
#pragma unroll
            for (int c = 0; c < 6; ++c) out_q2(s, c * 512 + l0, qout() + ((size_t)b * 6 + c) * TGV_BVOX + l0, qn[c]);
        }
    }
};


// Item sequences a CTA sweeps through: the first item, then next(i) until an item >= end.
// Strided runs (the level kernel): runs r = cta + m * grid of R consecutive items each.
// next() is called on each item in turn, so the position within the run is counted
// instead of taken modulo R.
struct StridedRuns {
    uint32_t R, G, end;
    uint32_t pos;  // position within its run of the item next() was last called on
    __device__ __forceinline__ uint32_t next(uint32_t i)
    {
        if (++pos < R) return i + 1;
        pos = 0;
        return i + 1 + (G - 1) * R;
    }
};
// One contiguous run of items [first, end) (a task of the batched kernel).
struct OneRun {
    uint32_t end;
    __device__ __forceinline__ uint32_t next(uint32_t i) { return i + 1; }
};

// Software-pipelined sweep of one CTA over the items first, q.next(first), ... < q.end
// (q.next is called on each item once, in order):
// in one barrier interval the CTA finishes item i (phase B) and starts the next item (its
// halo loads are issued first, so their latency overlaps phase B; then phase A once its
// stage has landed).  mbarriers 0 and 1 track the two stages; `parity` holds the phase
// each stage waits for next and carries over from one sweep to the next.  Returns false
// if a wait gave up: the domain's error flag is then set and the CTA's copies in flight
// have landed (so the caller may return).  `test_wait`: the first wait targets mbarrier
// 2, which nothing completes.
// ROLE 0: every thread owns a pair and a halo task (HW false); with HW, ROLE 1 is the own
// threads' sweep and ROLE 2 the halo warps' sweep.  The two roles run separate copies of the
// loop (so neither role's values are live across the other's code) that meet at the same
// sequence of CTA barriers.
template <int ROLE, typename S, typename D, int NB, bool HW, typename Seq>
__device__ __forceinline__ bool pair_sweep_role(PairCta<S, D, NB, HW>& C, Seq q, uint32_t it, uint32_t& parity,
                                                bool test_wait)
{
    using Cta = PairCta<S, D, NB, HW>;
    const PairArgs<S, D>& P = C.P;
    const uint32_t nit = q.end;
    const int32_t* work = C.A.work;
    const int* nbr = C.A.nbr;
    auto brick = [&](uint32_t i) -> uint32_t { return work ? (uint32_t)work[i] : i; };
    if (it >= nit) return true;
    uint64_t* bar = C.bar();
    const int t = C.t;
    // the thread that issues the stage copies (and, after a wait that gave up, drains
    // them): thread 0, or in the halo-warp form the first halo thread, so no own warp
    // spends the start of its interval on it
    const bool issuer = HW ? (ROLE == 2 && t == 256) : (t == 0);

    uint32_t itn = q.next(it);
    uint32_t bcur = brick(it), bnext = itn < nit ? brick(itn) : 0u;
    if (ROLE != 2 && t < TGV_NNBR) {
        C.nbr_row(0)[t] = nbr[(size_t)bcur * TGV_NNBR + t];
        if (itn < nit) C.nbr_row(1)[t] = nbr[(size_t)bnext * TGV_NNBR + t];
    }
    __syncthreads();
    uint32_t pending = 0;  // stages with copies in flight (thread 0's view)
    if (issuer) {
        fence_proxy_async_smem();  // earlier generic reads of the stages come first
        C.issue(0, bcur);
        pending = 1u;
        if (itn < nit) {
            C.issue(1, bnext);
            pending |= 2u;
        }
    }
    bool bail = false;
    int s = 0;
    // hand-over from the item in hand to the next one: the next item follows in the
    // same run and is this brick's +x neighbour (links are symmetric, so the next
    // brick's -x neighbour is this one)
    bool to_next = itn == it + 1 && itn < nit && C.nbr_row(0)[NB_PX] == (int)bnext;
    // prologue: phase A of the first item
    if constexpr (ROLE == 0) C.load_inputs(C.nbr_row(0), false, to_next);
    else if constexpr (ROLE == 1) C.load_own(C.nbr_row(0));
    else C.load_halo(C.nbr_row(0), C.task, C.tk, false, to_next);
    {
        const bool ok = test_wait ? mbar_wait_bounded(&bar[2], 0, P.wait_budget)
                                  : mbar_wait_bounded(&bar[0], parity & 1u, P.wait_budget);
        if (__syncthreads_or(!ok)) bail = true;
    }
    uint32_t links = 0;
    if (!bail) {
        parity ^= 1u;
        pending &= ~1u;
        if constexpr (ROLE == 0) links = C.phase_a(0, C.nbr_row(0), false, to_next, 0u);
        else if constexpr (ROLE == 1) links = C.phase_a_own(0, C.nbr_row(0), false, to_next, 0u);
        else C.halo_phase(0, C.nbr_row(0), false, to_next);
        __syncthreads();
    }
    while (!bail) {
        const int ns = s ^ 1;
        const uint32_t itnn = itn < nit ? q.next(itn) : nit;
        const uint32_t bnn = itnn < nit ? brick(itnn) : 0u;
        bool next_to_next = false;
        uint32_t next_links = 0;
        if (itn < nit) {
            next_to_next = itnn == itn + 1 && itnn < nit && C.nbr_row(ns)[NB_PX] == (int)bnn;
            if constexpr (ROLE == 0 && Cta::kEarlyLoads) C.load_inputs(C.nbr_row(ns), to_next, next_to_next);
        }
        // the row of the item in hand is no longer read (phase B takes its link bits): reuse
        // it for item itnn.  256 threads: threads 0-11 load and store it here; halo-warp
        // form: the first halo warp loads it here and stores it after issuing its face-task
        // loads (below), so the load's latency holds up no own warp
        if (ROLE == 0 && t < TGV_NNBR && itnn < nit) C.nbr_row(s)[t] = nbr[(size_t)bnn * TGV_NNBR + t];
        const bool nrow_hw = ROLE == 2 && t - 256 < TGV_NNBR && itnn < nit;
        const int nrow_v = nrow_hw ? nbr[(size_t)bnn * TGV_NNBR + t - 256] : 0;
        if constexpr (ROLE == 0) C.phase_b(s, bcur, links, to_next);
        if constexpr (ROLE == 1) C.phase_b(s, bcur, links, to_next, itn < nit ? C.nbr_row(ns) : nullptr);
        // halo warps: the next item's face-task inputs, while the own warps run phase B
        if constexpr (ROLE == 2) {
            if (itn < nit) C.load_halo(C.nbr_row(ns), C.task, C.tk, to_next, next_to_next);
            if (nrow_hw) C.nbr_row(s)[t - 256] = nrow_v;
        }
        bool late = false;
        if (itn < nit) {
            // no CTA barrier between phase B of this item and phase A of the next: they
            // work on different stages, except the hand-over slots of stage s (the -x
            // halo p slot and the parked partial sums of row (y, z)), which only lanes of
            // one warp share (a warp holds one z layer); a warp starts phase A once its
            // lanes are past phase B and the next stage has landed.  A wait that gives up
            // is agreed on at the barrier that closes the interval.
            const bool ok = mbar_wait_bounded(&bar[ns], (parity >> ns) & 1u, P.wait_budget);
            if (ok) {
                parity ^= 1u << ns;
                pending &= ~(1u << ns);
            }
            late = !ok;
            __syncwarp();
            if constexpr (ROLE == 0) {
                if (!Cta::kEarlyLoads) C.load_inputs(C.nbr_row(ns), to_next, next_to_next);
                next_links = C.phase_a(ns, C.nbr_row(ns), to_next, next_to_next, bcur);
            } else if constexpr (ROLE == 1) {
                next_links = C.phase_a_own(ns, C.nbr_row(ns), to_next, next_to_next, bcur);
            } else {
                C.halo_phase(ns, C.nbr_row(ns), to_next, next_to_next);
            }
        }
        // stage s, the phase A results of item itn and the hand-over are settled
        if (__syncthreads_or(late)) {
            bail = true;
            break;
        }
        if (issuer && itnn < nit) {
            fence_proxy_async_smem();
            C.issue(s, bnn);
            pending |= 1u << s;
        }
        if (itn >= nit) break;
        it = itn;
        itn = itnn;
        s = ns;
        links = next_links;
        bcur = bnext;
        bnext = bnn;
        to_next = next_to_next;
    }
    if (bail && issuer) {
        atomicExch(P.err, 1);
        // copies still in flight land before the CTA's shared memory is released (the
        // default budget, not the possibly tiny one of the wait that gave up)
        for (int k = 0; k < 2; ++k)
            if (pending & (1u << k)) mbar_wait_bounded(&bar[k], (parity >> k) & 1u, TGV_WAIT_CYCLES_DEFAULT);
    }
    return !bail;
}

template <typename S, typename D, int NB, bool HW, typename Seq>
__device__ __forceinline__ bool pair_sweep(PairCta<S, D, NB, HW>& C, Seq q, uint32_t it, uint32_t& parity,
                                           bool test_wait)
{
    if constexpr (!HW) return pair_sweep_role<0>(C, q, it, parity, test_wait);
    else if (C.own) return pair_sweep_role<1>(C, q, it, parity, test_wait);
    else return pair_sweep_role<2>(C, q, it, parity, test_wait);
}
