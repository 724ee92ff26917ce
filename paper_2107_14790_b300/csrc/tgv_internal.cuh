// Internal declarations of the TGV library (not part of the C-ABI).
//
// Device layout of one level (all arrays brick-major, 512 voxels per brick,
// local voxel index i + 8j + 64k):
//   bricks [0, nb) are active, [nb, nb + nf) frozen (Sec. 4.5, set B).
//   u      float [nb+nf][512]            (in place: only a voxel's own thread reads it)
//   ubar   float [2][nb+nf][512]         (ping-pong: neighbours read the old copy)
//   v      S     [nb+nf][3][512]         (in place)
//   vbar   S     [2][nb+nf][3][512]      (ping-pong)
//   p      S     [2][nb][3][512]         (ping-pong, active bricks only)
//   q      S     [2][nb][6][512]         (ping-pong; q_xx, q_yy, q_zz, q_xy, q_xz, q_yz)
//   hist   u32   [nb][npairs][512]       (bins 2k and 2k+1 as the low/high 16 bits)
//   nbr    int32 [nb][12]                (neighbour brick per slot; -1 = none;
//                                         index >= nb = frozen brick)
// S is float, __nv_bfloat16 or __half (the storage form of v, vbar, p, q).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "tgv.h"

#define TGV_BVOX 512
#define TGV_NNBR 12
#define TGV_MAX_BINS 16
#define TGV_MAPS_PER_LAUNCH 32
// default budget of a bounded device-side wait, in SM clock cycles (about one second)
#define TGV_WAIT_CYCLES_DEFAULT 2000000000LL

// budget of the iteration kernels' bounded waits for a domain's parameters
inline long long tgv_wait_budget(const tgv_params& p)
{
    return p.wait_cycles > 0 ? (long long)p.wait_cycles : TGV_WAIT_CYCLES_DEFAULT;
}

// Neighbour slots: the six faces, then the six edge bricks whose offset has
// -1 on one axis and +1 on another ("MX_PY" = offset (-1, +1, 0)).  The edge
// bricks are the only non-face bricks a fused iteration reads: the new dual
// at a -a face halo voxel needs ubar one step along +b, and the new q at a +a
// face halo voxel needs vbar one step along -b.
enum {
    NB_PX = 0, NB_MX = 1, NB_PY = 2, NB_MY = 3, NB_PZ = 4, NB_MZ = 5,
    NB_MX_PY = 6, NB_MX_PZ = 7, NB_MY_PX = 8, NB_MY_PZ = 9, NB_MZ_PX = 10, NB_MZ_PY = 11
};

__host__ __device__ inline int nb_plus(int a) { return 2 * a; }
__host__ __device__ inline int nb_minus(int a) { return 2 * a + 1; }
// slot of the edge brick with offset -1 on axis `m` and +1 on axis `p` (m != p)
__host__ __device__ inline int nb_edge(int m, int p)
{
    return 6 + 2 * m + (p > m ? p - 1 : p);
}

// ---------------------------------------------------------------- storage types
template <typename S> __device__ __forceinline__ float ld_s(const S* p);
template <> __device__ __forceinline__ float ld_s<float>(const float* p) { return *p; }
template <> __device__ __forceinline__ float ld_s<__nv_bfloat16>(const __nv_bfloat16* p) { return __bfloat162float(*p); }
template <> __device__ __forceinline__ float ld_s<__half>(const __half* p) { return __half2float(*p); }

template <typename S> __device__ __forceinline__ void st_s(S* p, float x);
template <> __device__ __forceinline__ void st_s<float>(float* p, float x) { *p = x; }
template <> __device__ __forceinline__ void st_s<__nv_bfloat16>(__nv_bfloat16* p, float x) { *p = __float2bfloat16_rn(x); }
template <> __device__ __forceinline__ void st_s<__half>(__half* p, float x) { *p = __float2half_rn(x); }

inline size_t storage_bytes(int storage) { return storage == TGV_STORAGE_FP32 ? 4 : 2; }

// ---------------------------------------------------------------- dual storage
// p and q are stored in the form's storage type, except in TGV_STORAGE_FX16: there they
// are 16-bit fixed point, the integer round(x * 32767 / bound) with bound = alpha1 for p
// and alpha0 for q (the radii of the balls the projections keep them in, so every
// component fits).  dsc = bound / 32767 decodes, isc = 32767 / bound encodes; both are
// ignored by the other storage types.
__device__ __forceinline__ int16_t fx16_encode(float x, float isc)
{
    const float y = fminf(fmaxf(__fmul_rn(x, isc), -32767.0f), 32767.0f);
    return (int16_t)__float2int_rn(y);
}
__device__ __forceinline__ float fx16_decode(int16_t i, float dsc) { return __fmul_rn((float)i, dsc); }
// Two values packed into one word (a low, b high) by the conversion to 16-bit integers,
// which saturates at [-32768, 32767]; equal to fx16_encode for |x| <= 32767.5 / isc, which
// holds for every dual the projections leave (|x| <= bound up to a few ulps).
__device__ __forceinline__ uint32_t fx16_encode2(float a, float b, float isc)
{
    uint32_t r;
    asm("{\n\t.reg .b16 lo, hi;\n\tcvt.rni.s16.f32 lo, %1;\n\tcvt.rni.s16.f32 hi, %2;\n\tmov.b32 %0, {lo, hi};\n\t}"
        : "=r"(r)
        : "f"(__fmul_rn(a, isc)), "f"(__fmul_rn(b, isc)));
    return r;
}

template <typename D> __device__ __forceinline__ float ld_d(const D* p, float /*dsc*/) { return ld_s(p); }
template <> __device__ __forceinline__ float ld_d<int16_t>(const int16_t* p, float dsc) { return fx16_decode(*p, dsc); }
template <typename D> __device__ __forceinline__ void st_d(D* p, float x, float /*isc*/) { st_s(p, x); }
template <> __device__ __forceinline__ void st_d<int16_t>(int16_t* p, float x, float isc) { *p = fx16_encode(x, isc); }

// decode / encode scales of p and q for a parameter set
struct DualScales {
    float dsp, dsq, isp, isq;
};
inline DualScales tgv_dual_scales(const tgv_params& prm)
{
    return {prm.alpha1 / 32767.0f, prm.alpha0 / 32767.0f, 32767.0f / prm.alpha1, 32767.0f / prm.alpha0};
}

// ---------------------------------------------------------------- host state
struct TgvLevel {
    int64_t nb = 0, nf = 0;  // active and frozen bricks
    double origin[3] = {0, 0, 0};
    double h = 1.0, radius = 0.5;
    std::vector<int32_t> coords;  // 3*(nb+nf), active first
    float* u = nullptr;
    float* ubar[2] = {nullptr, nullptr};
    void* v = nullptr;
    void* vbar[2] = {nullptr, nullptr};
    void* p[2] = {nullptr, nullptr};
    void* q[2] = {nullptr, nullptr};
    uint32_t* hist = nullptr;
    int32_t* nbr = nullptr;
    int32_t* coords_dev = nullptr;  // 3*(nb+nf) brick coordinates
    int32_t* work = nullptr;   // optional list of active bricks to update (device); nullptr = all
    int64_t nwork = 0;
    int64_t work_cap = 0;
    uint64_t work_gen = 0;     // bumped whenever the work list changes (invalidates cached graphs)
    struct Graph {
        int iters, parity;
        uint64_t gen;
        cudaGraphExec_t exec;
    };
    std::vector<Graph> graphs;
    // plans of the persistent batched solve (tgv_solve_chunks): device tables, and the
    // call captured as a CUDA graph when the domain has a stream
    struct Batch {
        uint64_t key = 0;
        void* dev = nullptr;
        size_t bytes = 0;
        cudaGraphExec_t exec = nullptr;
        int64_t launches = 0;  // kernels one replay launches
    };
    std::vector<Batch> batches;
    int cur = 0;               // ping-pong copy holding the current ubar/vbar/p/q
    uint64_t max_votes = 0;    // upper bound on any voxel's total count
    // host copies of nbr (nb rows) and of the work list, for the paired kernel's run-length choice
    std::vector<int32_t> nbr_host;
    std::vector<int32_t> work_host;
    int32_t* up7 = nullptr;    // marching cubes: nb x 7 upper-neighbour bricks (built on first use)
    int32_t* bgrid = nullptr;  // scatter-form histograms: active brick per cell of their bounding box
    int32_t bgmin[3] = {0, 0, 0}, bgdim[3] = {0, 0, 0};
    int xrun = 0;              // cached automatic run length, valid for (xrun_gen, xrun_slots)
    uint64_t xrun_gen = 0;
    int64_t xrun_slots = 0;
};

// Arguments of one fused primal-dual iteration over the active bricks of a level
// (S: storage type of v and vbar; D: of p and q).
template <typename S, typename D = S>
struct IterArgs {
    float* u;
    const float* ubar_in;
    float* ubar_out;
    S* v;
    const S* vbar_in;
    S* vbar_out;
    const D* p_in;
    D* p_out;
    const D* q_in;
    D* q_out;
    const uint32_t* hist;
    const int32_t* nbr;
    const int32_t* work;  // work item -> active brick (nullptr: item i is brick i)
    int64_t nitems;       // work items of this launch
    int64_t nb;    // active bricks (indices >= nb are frozen)
    int64_t nall;  // active + frozen bricks (stride of the in-place fields' brick index)
    int nbins, npairs, clamp_u;
    float alpha1, alpha0, tau, sigma, taulam;
    DualScales ds;          // fixed-point scales of p and q (TGV_STORAGE_FX16)
    float c[TGV_MAX_BINS];  // bin centres
};

struct TgvScratch {
    void* ptr = nullptr;
    size_t cap = 0;
};

struct tgv_domain {
    std::vector<TgvLevel> levels;
    tgv_params prm{};
    cudaStream_t stream = nullptr;
    int device = 0;
    int sm_count = 0;
    bool broken = false;
    std::string last_error;
    int64_t launches = 0;
    int64_t bytes = 0;
    TgvScratch pyr;     // depth pyramids of one accumulation batch
    TgvScratch red;     // per-block partial sums of the energy reduction
    TgvScratch tmp;     // staging for host <-> device field copies
    TgvScratch table;   // per-brick parent table of tgv_prolong
    TgvScratch mesh_flags, mesh_count, mesh_cells, mesh_scan, mesh_v, mesh_t;  // marching cubes
    int64_t mesh_nv = -1, mesh_nt = -1;  // counts of the last extracted mesh (-1: none)
    double* red_out = nullptr;   // 4 doubles: final reduction result (device)
    int* err = nullptr;          // device flag: 1 after a bounded device-side wait gave up
};

// Sets the kernel's dynamic shared memory limit and returns its CTAs per SM
// (cached per kernel, block size and shared memory size; safe to call while a
// stream is being captured once the first call has happened outside capture).
tgv_status tgv_kernel_setup(const void* kernel, int threads, size_t smem, int* per_sm);

// Makes `dev` the current device for the guard's lifetime.
struct DeviceGuard {
    int old = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&old) == cudaSuccess && old != dev) cudaSetDevice(dev);
        else old = -1;
    }
    ~DeviceGuard()
    {
        if (old >= 0) cudaSetDevice(old);
    }
};

// helpers implemented in tgv_domain.cu
tgv_status tgv_fail(tgv_domain* d, tgv_status s, const std::string& msg);
// INVALID_ARG for NULL, STATE for a domain broken by an earlier error, else OK
tgv_status tgv_check_domain(tgv_domain* d);
tgv_status tgv_cuda_check(tgv_domain* d, cudaError_t e, const char* what);
tgv_status tgv_scratch(tgv_domain* d, TgvScratch& s, size_t bytes);
void tgv_bin_centres(const tgv_params& prm, float* c);

// Marching cubes of level L into the domain's mesh buffers (synchronises).
tgv_status tgv_mesh_extract(tgv_domain* d, TgvLevel& L, int64_t* nverts, int64_t* ntris);
// CTAs (= partial sums) of the energy kernel for nitems bricks: sixteen per SM of the
// current device, at most nitems
int64_t tgv_energy_grid(int64_t nitems);
// exclusive prefix sum of n counts in place on the domain's stream (its tile sums in
// tmp); *total = the sum (synchronises).  Sums must stay below 2^32.
tgv_status tgv_exclusive_scan_u32(tgv_domain* d, uint32_t* data, int64_t n, TgvScratch& tmp, uint64_t* total);

// Number of bricks one iteration updates.
inline int64_t tgv_work_items(const TgvLevel& L) { return L.work ? L.nwork : L.nb; }

// Iteration arguments for the current ping-pong copy of a level.
template <typename S, typename D = S>
inline IterArgs<S, D> tgv_make_iter_args(tgv_domain* d, TgvLevel& L)
{
    IterArgs<S, D> A;
    const int c = L.cur, o = 1 - L.cur;
    A.u = L.u;
    A.ubar_in = L.ubar[c];
    A.ubar_out = L.ubar[o];
    A.v = (S*)L.v;
    A.vbar_in = (const S*)L.vbar[c];
    A.vbar_out = (S*)L.vbar[o];
    A.p_in = (const D*)L.p[c];
    A.p_out = (D*)L.p[o];
    A.q_in = (const D*)L.q[c];
    A.q_out = (D*)L.q[o];
    A.hist = L.hist;
    A.nbr = L.nbr;
    A.work = L.work;
    A.nitems = L.work ? L.nwork : L.nb;
    A.nb = L.nb;
    A.nall = L.nb + L.nf;
    A.nbins = d->prm.nbins;
    A.npairs = (d->prm.nbins + 1) / 2;
    A.clamp_u = d->prm.clamp_u;
    A.alpha1 = d->prm.alpha1;
    A.alpha0 = d->prm.alpha0;
    A.tau = d->prm.tau;
    A.sigma = d->prm.sigma;
    A.taulam = d->prm.tau * d->prm.lambda;
    A.ds = tgv_dual_scales(d->prm);
    tgv_bin_centres(d->prm, A.c);
    return A;
}

// serving-engine helpers implemented in tgv_domain.cu
tgv_status tgv_create_arena(const tgv_params* prm, cudaStream_t stream, int64_t cap_active, int64_t cap_frozen,
                            tgv_domain** out);
void tgv_launch_f32_to_storage(tgv_domain* d, const float* src, void* dst, int64_t n);
void tgv_launch_hist_pack(tgv_domain* d, uint32_t* dst, const uint32_t* src, int64_t nvox, unsigned int* maxc);

// launchers implemented in tgv_solve.cu / tgv_iter_pipe.cu / tgv_hist.cu
tgv_status tgv_launch_iterations(tgv_domain* d, TgvLevel& L, int iters);
tgv_status tgv_launch_iterations_pipe(tgv_domain* d, TgvLevel& L, int iters);
bool tgv_pipe_supports(const TgvLevel& L);
tgv_status tgv_launch_iterations_pair(tgv_domain* d, TgvLevel& L, int iters);
tgv_status tgv_check_device_error(tgv_domain* d);
tgv_status tgv_launch_energy(tgv_domain* d, TgvLevel& L, double* host_out);
cudaError_t tgv_launch_energy_view(const tgv_state_view& s, const tgv_params& prm, cudaStream_t stream,
                                   double* partial, double* result);
tgv_status tgv_launch_accumulate(tgv_domain* d, TgvLevel& L, const tgv_camera* cams, int nmaps,
                                 const float* depth, int64_t pitch, int64_t stride, const uint32_t* votes);
