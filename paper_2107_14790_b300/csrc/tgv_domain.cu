// Host side of the C-ABI declared in include/tgv.h: domain creation (brick
// neighbour tables, device state), field and histogram transfers, reset,
// coarse-to-fine prolongation, error handling.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <unordered_map>

#include "tgv_internal.cuh"
#include "tgv_nvtx.h"

// ------------------------------------------------------------------------- errors
tgv_status tgv_fail(tgv_domain* d, tgv_status s, const std::string& msg)
{
    if (d) d->last_error = msg;
    return s;
}

tgv_status tgv_cuda_check(tgv_domain* d, cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return TGV_OK;
    if (d) {
        d->broken = true;
        d->last_error = std::string(what) + ": " + cudaGetErrorString(e);
    }
    return TGV_ERR_CUDA;
}

// Reads the device error flag (the stream must be synchronised by the caller).
tgv_status tgv_check_device_error(tgv_domain* d)
{
    int flag = 0;
    cudaError_t e = cudaMemcpy(&flag, d->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return tgv_cuda_check(d, e, "error flag read");
    if (flag) {
        d->broken = true;
        d->last_error = "a bounded device-side wait gave up (pipelined iteration kernel)";
        return TGV_ERR_TIMEOUT;
    }
    return TGV_OK;
}

tgv_status tgv_kernel_setup(const void* kernel, int threads, size_t smem, int* per_sm)
{
    static std::mutex mu;
    static std::map<std::tuple<const void*, int, int, size_t>, int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TGV_ERR_CUDA;
    std::lock_guard<std::mutex> lock(mu);
    auto key = std::make_tuple(kernel, dev, threads, smem);
    auto it = cache.find(key);
    if (it != cache.end()) {
        *per_sm = it->second;
        return TGV_OK;
    }
    // The limit is raised to the device maximum (less the kernel's static shared memory,
    // not to `smem`): the same kernel may be
    // launched with different shared-memory sizes, and a lower limit set for one
    // size would make launches with a larger one fail.
    int optin = 0;
    cudaFuncAttributes fa;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) {
        cudaGetLastError();
        return TGV_ERR_CUDA;
    }
    const int dyn_max = optin - (int)fa.sharedSizeBytes;  // the kernel's static shared memory counts too
    if (dyn_max < 0 || (size_t)dyn_max < smem ||
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kernel, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return TGV_ERR_CUDA;
    }
    cache[key] = *per_sm;
    return TGV_OK;
}

tgv_status tgv_scratch(tgv_domain* d, TgvScratch& s, size_t bytes)
{
    if (bytes <= s.cap) return TGV_OK;
    if (s.ptr) {
        // the old buffer may still be read by queued work
        cudaError_t e = cudaStreamSynchronize(d->stream);
        if (e != cudaSuccess) return tgv_cuda_check(d, e, "scratch sync");
        cudaFree(s.ptr);
        d->bytes -= (int64_t)s.cap;
        s.ptr = nullptr;
        s.cap = 0;
    }
    size_t cap = std::max(bytes, (size_t)1 << 20);
    cudaError_t e = cudaMalloc(&s.ptr, cap);
    if (e != cudaSuccess) {
        cudaGetLastError();
        s.ptr = nullptr;
        return tgv_fail(d, TGV_ERR_OUT_OF_MEMORY, "scratch allocation failed");
    }
    s.cap = cap;
    d->bytes += (int64_t)cap;
    return TGV_OK;
}

void tgv_bin_centres(const tgv_params& prm, float* c)
{
    const int n = prm.nbins;
    for (int b = 0; b < TGV_MAX_BINS; ++b) {
        double v = 0.0;
        if (b < n)
            v = prm.centres == TGV_CENTRES_ENDPOINTS ? -1.0 + 2.0 * b / (double)(n - 1)
                                                     : -1.0 + (2.0 * b + 1.0) / (double)n;
        c[b] = (float)v;
    }
}

namespace {

inline uint64_t brick_key(int32_t x, int32_t y, int32_t z)
{
    const uint64_t B = (uint64_t)1 << 20;
    return (((uint64_t)(z + (int64_t)B) * (2 * B)) + (uint64_t)(y + (int64_t)B)) * (2 * B) + (uint64_t)(x + (int64_t)B);
}

const int kSlotOffset[TGV_NNBR][3] = {
    {+1, 0, 0}, {-1, 0, 0}, {0, +1, 0}, {0, -1, 0}, {0, 0, +1}, {0, 0, -1},
    {-1, +1, 0}, {-1, 0, +1}, {+1, -1, 0}, {0, -1, +1}, {+1, 0, -1}, {0, +1, -1}};

int ncomp_of(int field)
{
    switch (field) {
    case TGV_FIELD_U:
    case TGV_FIELD_UBAR: return 1;
    case TGV_FIELD_V:
    case TGV_FIELD_VBAR:
    case TGV_FIELD_P: return 3;
    case TGV_FIELD_Q: return 6;
    }
    return 0;
}

bool is_device_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

unsigned grid1(int64_t n, int block, int sms)
{
    int64_t g = (n + block - 1) / block;
    int64_t cap = (int64_t)sms * 32;
    if (g > cap) g = cap;
    return (unsigned)std::max<int64_t>(g, 1);
}

// ------------------------------------------------------------------------- kernels
template <typename S>
__global__ void f32_to_s_kernel(const float* __restrict__ src, S* __restrict__ dst, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        st_s(dst + i, src[i]);
}

// brick-major [brick][comp][512] storage <-> voxel-major [voxel][comp] float
// (sc: decode scale of fixed-point duals, ignored by the other storage types)
template <typename S>
__global__ void field_extract_kernel(const S* __restrict__ f, float* __restrict__ out, int64_t nvox, int ncomp,
                                     float sc)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvox * ncomp;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t vox = i / ncomp;
        const int c = (int)(i - vox * ncomp);
        const int64_t b = vox >> 9, l = vox & 511;
        out[i] = ld_d(f + (b * ncomp + c) * TGV_BVOX + l, sc);
    }
}

// (sc: encode scale of fixed-point duals, ignored by the other storage types)
template <typename S>
__global__ void field_set_kernel(S* __restrict__ f, const float* __restrict__ in, int64_t nvox, int ncomp, float sc)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvox * ncomp;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t vox = i / ncomp;
        const int c = (int)(i - vox * ncomp);
        const int64_t b = vox >> 9, l = vox & 511;
        st_d(f + (b * ncomp + c) * TGV_BVOX + l, in[i], sc);
    }
}

__global__ void hist_unpack_kernel(const uint32_t* __restrict__ h, uint32_t* __restrict__ out, int64_t nvox, int nbins,
                                   int npairs)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvox * nbins;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t vox = i / nbins;
        const int k = (int)(i - vox * nbins);
        const int64_t b = vox >> 9, l = vox & 511;
        const uint32_t w = h[(b * npairs + (k >> 1)) * TGV_BVOX + l];
        out[i] = (w >> ((k & 1) * 16)) & 0xffffu;
    }
}

// one thread per (voxel, pair); records the largest input count in *maxc
__global__ void hist_pack_kernel(uint32_t* __restrict__ h, const uint32_t* __restrict__ in, int64_t nvox, int nbins,
                                 int npairs, unsigned int* maxc)
{
    unsigned int m = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvox * npairs;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t vox = i / npairs;
        const int k = (int)(i - vox * npairs);
        const int64_t b = vox >> 9, l = vox & 511;
        const uint32_t lo = in[vox * nbins + 2 * k];
        const uint32_t hi = 2 * k + 1 < nbins ? in[vox * nbins + 2 * k + 1] : 0u;
        m = max(m, max(lo, hi));
        h[(b * npairs + k) * TGV_BVOX + l] = (lo & 0xffffu) | ((hi & 0xffffu) << 16);
    }
    if (m) atomicMax(maxc, m);
}

// Fine voxel (brick fb, local l) takes u and v/2 of its parent voxel; all 512
// voxels of a fine brick share one parent brick (parent[fb], -1 = none).
template <typename S>
__global__ void prolong_kernel(const float* __restrict__ cu, const S* __restrict__ cv, const int32_t* __restrict__ parent,
                               const int32_t* __restrict__ fcoords, int64_t nfall, int64_t nfact, float* fu,
                               float* fub0, float* fub1, S* fv, S* fvb0, S* fvb1)
{
    const int64_t fb = blockIdx.x;
    const int l = threadIdx.x;
    const int loc[3] = {l & 7, (l >> 3) & 7, l >> 6};
    const int32_t pb = parent[fb];
    float u = 0.0f, v[3] = {0.0f, 0.0f, 0.0f};
    if (pb >= 0) {
        int cl[3];
        for (int a = 0; a < 3; ++a) cl[a] = 4 * (fcoords[3 * fb + a] & 1) + (loc[a] >> 1);
        const int64_t ci = (int64_t)cl[0] + 8 * cl[1] + 64 * cl[2];
        u = cu[(int64_t)pb * TGV_BVOX + ci];
        for (int c = 0; c < 3; ++c) v[c] = 0.5f * ld_s(cv + ((int64_t)pb * 3 + c) * TGV_BVOX + ci);
    }
    const int64_t vi = fb * TGV_BVOX + l;
    fu[vi] = u;
    fub0[vi] = u;
    fub1[vi] = u;
    for (int c = 0; c < 3; ++c) {
        const int64_t oi = (fb * 3 + c) * TGV_BVOX + l;
        st_s(fv + oi, v[c]);
        st_s(fvb0 + oi, v[c]);
        st_s(fvb1 + oi, v[c]);
    }
    (void)nfall;
    (void)nfact;
}

tgv_status check_domain(tgv_domain* d)
{
    if (!d) return TGV_ERR_INVALID_ARG;
    if (d->broken) return tgv_fail(d, TGV_ERR_STATE, "domain unusable after an earlier CUDA error: " + d->last_error);
    return TGV_OK;
}

}  // namespace

tgv_status tgv_check_domain(tgv_domain* d) { return check_domain(d); }

namespace {

tgv_status get_level(tgv_domain* d, int32_t level, TgvLevel** L)
{
    if (level < 0 || level >= (int32_t)d->levels.size()) return tgv_fail(d, TGV_ERR_INVALID_ARG, "level out of range");
    *L = &d->levels[level];
    return TGV_OK;
}

tgv_status dalloc(tgv_domain* d, void** p, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return tgv_fail(d, TGV_ERR_OUT_OF_MEMORY, "device allocation of " + std::to_string(bytes) + " bytes failed");
    }
    d->bytes += (int64_t)bytes;
    return TGV_OK;
}

void free_graphs(TgvLevel& L)
{
    for (auto& g : L.graphs) cudaGraphExecDestroy(g.exec);
    L.graphs.clear();
    for (auto& b : L.batches) {
        if (b.exec) cudaGraphExecDestroy(b.exec);
        if (b.dev) cudaFree(b.dev);
    }
    L.batches.clear();
}

void free_level(TgvLevel& L)
{
    free_graphs(L);
    void* ptrs[] = {L.u, L.ubar[0], L.ubar[1], L.v, L.vbar[0], L.vbar[1], L.p[0], L.p[1],
                    L.q[0], L.q[1], L.hist, L.nbr, L.coords_dev, L.work, L.up7, L.bgrid};
    for (void* p : ptrs)
        if (p) cudaFree(p);
}

void* field_ptr(TgvLevel& L, int field)
{
    switch (field) {
    case TGV_FIELD_U: return L.u;
    case TGV_FIELD_UBAR: return L.ubar[L.cur];
    case TGV_FIELD_V: return L.v;
    case TGV_FIELD_VBAR: return L.vbar[L.cur];
    case TGV_FIELD_P: return L.p[L.cur];
    case TGV_FIELD_Q: return L.q[L.cur];
    }
    return nullptr;
}

template <typename S>
void launch_f32_to_s(tgv_domain* d, const float* src, void* dst, int64_t n)
{
    f32_to_s_kernel<S><<<grid1(n, 256, d->sm_count), 256, 0, d->stream>>>(src, (S*)dst, n);
    d->launches++;
}

void f32_to_storage(tgv_domain* d, const float* src, void* dst, int64_t n)
{
    switch (d->prm.storage) {
    case TGV_STORAGE_FP32: launch_f32_to_s<float>(d, src, dst, n); break;
    case TGV_STORAGE_BF16: launch_f32_to_s<__nv_bfloat16>(d, src, dst, n); break;
    default: launch_f32_to_s<__half>(d, src, dst, n); break;
    }
}

// Allocates and zeroes every array of a level with nb active and nf frozen
// bricks (neighbour table: all "none"; coordinates: zero).
tgv_status alloc_level(tgv_domain* d, TgvLevel& L, int64_t nb, int64_t nf)
{
    L.nb = nb;
    L.nf = nf;
    const int64_t na = nb + nf;
    const size_t sb = storage_bytes(d->prm.storage);
    const int npairs = (d->prm.nbins + 1) / 2;
    const size_t va = (size_t)na * TGV_BVOX, vn = (size_t)nb * TGV_BVOX;
    tgv_status st = TGV_OK;
    void** fl[] = {(void**)&L.u, (void**)&L.ubar[0], (void**)&L.ubar[1]};
    for (void** p : fl)
        if ((st = dalloc(d, p, va * 4)) != TGV_OK) return st;
    void** vl[] = {&L.v, &L.vbar[0], &L.vbar[1]};
    for (void** p : vl)
        if ((st = dalloc(d, p, 3 * va * sb)) != TGV_OK) return st;
    for (int k = 0; k < 2; ++k) {
        if ((st = dalloc(d, &L.p[k], 3 * vn * sb)) != TGV_OK) return st;
        if ((st = dalloc(d, &L.q[k], 6 * vn * sb)) != TGV_OK) return st;
    }
    if ((st = dalloc(d, (void**)&L.hist, (size_t)npairs * vn * 4)) != TGV_OK) return st;
    if ((st = dalloc(d, (void**)&L.nbr, (size_t)nb * TGV_NNBR * 4)) != TGV_OK) return st;
    if ((st = dalloc(d, (void**)&L.coords_dev, (size_t)na * 3 * 4)) != TGV_OK) return st;
    cudaStream_t s = d->stream;
    cudaError_t e = cudaMemsetAsync(L.u, 0, va * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(L.ubar[0], 0, va * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(L.ubar[1], 0, va * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(L.v, 0, 3 * va * sb, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(L.vbar[0], 0, 3 * va * sb, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(L.vbar[1], 0, 3 * va * sb, s);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaMemsetAsync(L.p[k], 0, 3 * vn * sb, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(L.q[k], 0, 6 * vn * sb, s);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(L.hist, 0, (size_t)npairs * vn * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(L.nbr, 0xff, (size_t)nb * TGV_NNBR * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(L.coords_dev, 0, (size_t)na * 3 * 4, s);
    return tgv_cuda_check(d, e, "level allocation");
}

tgv_status build_level(tgv_domain* d, const tgv_level_desc& desc, TgvLevel& L)
{
    if (desc.nbricks < 0 || desc.nfrozen < 0 || (desc.nbricks > 0 && !desc.brick_coords) ||
        (desc.nfrozen > 0 && !desc.frozen_coords))
        return tgv_fail(d, TGV_ERR_INVALID_ARG, "bad brick list");
    if (!(desc.h > 0.0) || !isfinite(desc.h)) return tgv_fail(d, TGV_ERR_INVALID_ARG, "h must be positive");
    const int64_t nb = desc.nbricks, nf = desc.nfrozen, na = nb + nf;
    if (na > ((int64_t)1 << 31) / 2) return tgv_fail(d, TGV_ERR_INVALID_ARG, "too many bricks");
    L.nb = nb;
    L.nf = nf;
    for (int a = 0; a < 3; ++a) L.origin[a] = desc.origin[a];
    L.h = desc.h;
    L.radius = desc.radius > 0.0 ? desc.radius : desc.h / 2.0;
    L.coords.resize(3 * (size_t)na);
    std::unordered_map<uint64_t, int32_t> index;
    index.reserve((size_t)na * 2);
    for (int64_t i = 0; i < na; ++i) {
        const int32_t* c = i < nb ? desc.brick_coords + 3 * i : desc.frozen_coords + 3 * (i - nb);
        for (int a = 0; a < 3; ++a) {
            if (c[a] < -(1 << 19) || c[a] >= (1 << 19))
                return tgv_fail(d, TGV_ERR_INVALID_ARG, "brick coordinate out of range");
            L.coords[3 * i + a] = c[a];
        }
        if (!index.emplace(brick_key(c[0], c[1], c[2]), (int32_t)i).second)
            return tgv_fail(d, TGV_ERR_INVALID_ARG, "duplicate brick coordinates");
    }
    std::vector<int32_t> nbr((size_t)nb * TGV_NNBR);
    for (int64_t i = 0; i < nb; ++i)
        for (int s = 0; s < TGV_NNBR; ++s) {
            auto it = index.find(brick_key(L.coords[3 * i] + kSlotOffset[s][0], L.coords[3 * i + 1] + kSlotOffset[s][1],
                                           L.coords[3 * i + 2] + kSlotOffset[s][2]));
            nbr[(size_t)i * TGV_NNBR + s] = it == index.end() ? -1 : it->second;
        }
    const size_t sb = storage_bytes(d->prm.storage);
    const size_t vn = (size_t)nb * TGV_BVOX;
    tgv_status st = alloc_level(d, L, nb, nf);
    if (st != TGV_OK) return st;
    cudaStream_t s = d->stream;
    cudaError_t e = cudaSuccess;
    if (!nbr.empty()) e = cudaMemcpyAsync(L.nbr, nbr.data(), nbr.size() * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !L.coords.empty())
        e = cudaMemcpyAsync(L.coords_dev, L.coords.data(), L.coords.size() * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // host vectors above are about to go away
    if ((st = tgv_cuda_check(d, e, "level initialisation")) != TGV_OK) return st;
    L.nbr_host = std::move(nbr);
    // frozen values (set B): constant u and v, mirrored into both ping-pong copies
    if (nf > 0 && desc.frozen_u) {
        const size_t n = (size_t)nf * TGV_BVOX;
        for (float* dst : {L.u, L.ubar[0], L.ubar[1]}) {
            e = cudaMemcpyAsync(dst + vn, desc.frozen_u, n * 4, cudaMemcpyHostToDevice, s);
            if ((st = tgv_cuda_check(d, e, "frozen u upload")) != TGV_OK) return st;
        }
    }
    if (nf > 0 && desc.frozen_v) {
        const size_t n = 3 * (size_t)nf * TGV_BVOX;
        if ((st = tgv_scratch(d, d->tmp, n * 4)) != TGV_OK) return st;
        e = cudaMemcpyAsync(d->tmp.ptr, desc.frozen_v, n * 4, cudaMemcpyHostToDevice, s);
        if ((st = tgv_cuda_check(d, e, "frozen v upload")) != TGV_OK) return st;
        for (void* dst : {L.v, L.vbar[0], L.vbar[1]})
            f32_to_storage(d, (const float*)d->tmp.ptr, (char*)dst + 3 * vn * sb, (int64_t)n);
        e = cudaStreamSynchronize(s);
        if ((st = tgv_cuda_check(d, e, "frozen v conversion")) != TGV_OK) return st;
    }
    return TGV_OK;
}

}  // namespace

// ---- helpers used by the serving engine (tgv_server.cu)
tgv_status tgv_create_arena(const tgv_params* prm, cudaStream_t stream, int64_t cap_active, int64_t cap_frozen,
                            tgv_domain** out)
{
    *out = nullptr;
    tgv_domain* d = new (std::nothrow) tgv_domain();
    if (!d) return TGV_ERR_OUT_OF_MEMORY;
    d->prm = *prm;
    d->stream = stream;
    cudaError_t e = cudaGetDevice(&d->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&d->sm_count, cudaDevAttrMultiProcessorCount, d->device);
    tgv_status st = tgv_cuda_check(d, e, "device query");
    if (st == TGV_OK) st = dalloc(d, (void**)&d->red_out, 4 * sizeof(double));
    if (st == TGV_OK) st = dalloc(d, (void**)&d->err, sizeof(int));
    if (st == TGV_OK) st = tgv_cuda_check(d, cudaMemsetAsync(d->err, 0, sizeof(int), d->stream), "error flag");
    d->levels.resize(1);
    if (st == TGV_OK) st = alloc_level(d, d->levels[0], cap_active, cap_frozen);
    if (st == TGV_OK) d->levels[0].nbr_host.assign((size_t)cap_active * TGV_NNBR, -1);
    if (st == TGV_OK) st = tgv_cuda_check(d, cudaStreamSynchronize(d->stream), "arena initialisation");
    if (st != TGV_OK) {
        tgv_destroy_domain(d);
        return st;
    }
    *out = d;
    return TGV_OK;
}

void tgv_launch_f32_to_storage(tgv_domain* d, const float* src, void* dst, int64_t n) { f32_to_storage(d, src, dst, n); }

void tgv_launch_hist_pack(tgv_domain* d, uint32_t* dst, const uint32_t* src, int64_t nvox, unsigned int* maxc)
{
    const int npairs = (d->prm.nbins + 1) / 2;
    hist_pack_kernel<<<grid1(nvox * npairs, 256, d->sm_count), 256, 0, d->stream>>>(dst, src, nvox, d->prm.nbins,
                                                                                  npairs, maxc);
    d->launches++;
}

// ========================================================================= C-ABI
extern "C" {

const char* tgv_status_string(tgv_status s)
{
    switch (s) {
    case TGV_OK: return "ok";
    case TGV_ERR_INVALID_ARG: return "invalid argument";
    case TGV_ERR_OUT_OF_MEMORY: return "out of memory";
    case TGV_ERR_BUDGET: return "budget exceeded";
    case TGV_ERR_CUDA: return "CUDA error";
    case TGV_ERR_TIMEOUT: return "device wait timed out";
    case TGV_ERR_STATE: return "domain in error state";
    case TGV_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char* tgv_last_error(const tgv_domain* d) { return d ? d->last_error.c_str() : "null domain"; }

tgv_status tgv_default_params(tgv_params* out)
{
    if (!out) return TGV_ERR_INVALID_ARG;
    out->nbins = 8;
    out->alpha1 = 1.0f;
    out->alpha0 = 2.0f;
    out->lambda = 1.0f;
    out->tau = 0.2f;
    out->sigma = 0.2f;
    out->storage = TGV_STORAGE_FP32;
    out->clamp_u = 1;
    out->centres = TGV_CENTRES_ENDPOINTS;
    out->box_v = 2.0f;
    out->iter_kernel = TGV_ITER_PAIRED;
    out->x_run = 0;
    out->hist_form = TGV_HIST_GATHER;
    out->wait_cycles = 0;
    out->wait_test = 0;
    return TGV_OK;
}

tgv_status tgv_create_domain(const tgv_level_desc* levels, int32_t nlevels, const tgv_params* prm, void* stream,
                             tgv_domain** out)
{
    if (!out) return TGV_ERR_INVALID_ARG;
    *out = nullptr;
    if (!levels || nlevels <= 0 || nlevels > 32 || !prm) return TGV_ERR_INVALID_ARG;
    if (prm->nbins < 2 || prm->nbins > TGV_MAX_BINS) return TGV_ERR_INVALID_ARG;
    if (prm->storage < TGV_STORAGE_FP32 || prm->storage > TGV_STORAGE_FX16) return TGV_ERR_INVALID_ARG;
    if (prm->centres != TGV_CENTRES_ENDPOINTS && prm->centres != TGV_CENTRES_MIDPOINTS) return TGV_ERR_INVALID_ARG;
    if (prm->iter_kernel != TGV_ITER_PIPELINED && prm->iter_kernel != TGV_ITER_ONE_BRICK_PER_CTA &&
        prm->iter_kernel != TGV_ITER_PAIRED)
        return TGV_ERR_INVALID_ARG;
    if (prm->x_run < 0 || prm->x_run > 64) return TGV_ERR_INVALID_ARG;
    if (prm->hist_form != TGV_HIST_GATHER && prm->hist_form != TGV_HIST_SCATTER) return TGV_ERR_INVALID_ARG;
    if (prm->wait_cycles < 0 || (prm->wait_test != 0 && prm->wait_test != 1)) return TGV_ERR_INVALID_ARG;
    if (!(prm->alpha1 > 0.0f) || !(prm->alpha0 > 0.0f) || !(prm->lambda >= 0.0f) || !(prm->tau > 0.0f) ||
        !(prm->sigma > 0.0f) || !(prm->box_v > 0.0f))
        return TGV_ERR_INVALID_ARG;
    tgv_domain* d = new (std::nothrow) tgv_domain();
    if (!d) return TGV_ERR_OUT_OF_MEMORY;
    d->prm = *prm;
    d->stream = (cudaStream_t)stream;
    cudaError_t e = cudaGetDevice(&d->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&d->sm_count, cudaDevAttrMultiProcessorCount, d->device);
    tgv_status st = tgv_cuda_check(d, e, "device query");
    if (st == TGV_OK) st = dalloc(d, (void**)&d->red_out, 4 * sizeof(double));
    if (st == TGV_OK) st = dalloc(d, (void**)&d->err, sizeof(int));
    if (st == TGV_OK) st = tgv_cuda_check(d, cudaMemsetAsync(d->err, 0, sizeof(int), d->stream), "error flag");
    d->levels.resize((size_t)nlevels);
    for (int32_t l = 0; l < nlevels && st == TGV_OK; ++l) st = build_level(d, levels[l], d->levels[l]);
    if (st != TGV_OK) {
        std::string msg = d->last_error;
        tgv_destroy_domain(d);
        (void)msg;
        return st;
    }
    *out = d;
    return TGV_OK;
}

void tgv_destroy_domain(tgv_domain* d)
{
    if (!d) return;
    DeviceGuard g(d->device);
    cudaStreamSynchronize(d->stream);
    for (TgvLevel& L : d->levels) free_level(L);
    for (TgvScratch* s : {&d->pyr, &d->red, &d->tmp, &d->table, &d->mesh_flags, &d->mesh_count, &d->mesh_cells,
                          &d->mesh_scan, &d->mesh_v, &d->mesh_t})
        if (s->ptr) cudaFree(s->ptr);
    if (d->red_out) cudaFree(d->red_out);
    if (d->err) cudaFree(d->err);
    cudaGetLastError();
    delete d;
}

tgv_status tgv_accumulate_depthmaps(tgv_domain* d, int32_t level, const tgv_camera* cams, int32_t nmaps,
                                    const float* depth_dev, int64_t pitch_elems, int64_t map_stride_elems,
                                    const uint32_t* votes)
{
    TgvNvtxRange nvtx_range_("tgv_accumulate_depthmaps");
    tgv_status st = check_domain(d);
    if (st != TGV_OK) return st;
    DeviceGuard g(d->device);
    TgvLevel* L;
    if ((st = get_level(d, level, &L)) != TGV_OK) return st;
    if (nmaps < 0 || (nmaps > 0 && (!cams || !depth_dev))) return tgv_fail(d, TGV_ERR_INVALID_ARG, "bad map batch");
    if (nmaps == 0) return TGV_OK;
    const int W = cams[0].width, H = cams[0].height;
    if (W <= 0 || H <= 0 || W > 32768 || H > 32768) return tgv_fail(d, TGV_ERR_INVALID_ARG, "bad map size");
    if (pitch_elems < W) return tgv_fail(d, TGV_ERR_INVALID_ARG, "pitch smaller than width");
    if (nmaps > 1 && map_stride_elems < pitch_elems * H) return tgv_fail(d, TGV_ERR_INVALID_ARG, "map stride too small");
    uint64_t add = 0;
    for (int m = 0; m < nmaps; ++m) {
        const tgv_camera& c = cams[m];
        if (c.width != W || c.height != H) return tgv_fail(d, TGV_ERR_INVALID_ARG, "maps of one batch differ in size");
        if (c.model != TGV_PINHOLE && c.model != TGV_SPHERICAL) return tgv_fail(d, TGV_ERR_INVALID_ARG, "unknown camera model");
        bool ok = isfinite(c.fx) && isfinite(c.fy) && isfinite(c.cx) && isfinite(c.cy) && c.fx > 0 && c.fy > 0;
        for (int k = 0; k < 9; ++k) ok = ok && isfinite(c.R[k]);
        for (int k = 0; k < 3; ++k) ok = ok && isfinite(c.C[k]);
        if (!ok) return tgv_fail(d, TGV_ERR_INVALID_ARG, "camera parameters must be finite, fx and fy positive");
        const uint32_t v = votes ? votes[m] : 1u;
        if (v == 0 || v > 65535) return tgv_fail(d, TGV_ERR_INVALID_ARG, "vote must be in 1..65535");
        add += v;
    }
    if (L->max_votes + add > 65535)
        return tgv_fail(d, TGV_ERR_BUDGET, "a histogram count could exceed 65535 (16-bit bins)");
    if (L->nb == 0) return TGV_OK;
    st = tgv_launch_accumulate(d, *L, cams, nmaps, depth_dev, pitch_elems, nmaps > 1 ? map_stride_elems : 0, votes);
    if (st == TGV_OK) L->max_votes += add;
    return st;
}

tgv_status tgv_accumulate_depthmap(tgv_domain* d, int32_t level, const tgv_camera* cam, const float* depth_dev,
                                   int64_t pitch_elems, uint32_t vote)
{
    return tgv_accumulate_depthmaps(d, level, cam, 1, depth_dev, pitch_elems, 0, &vote);
}

tgv_status tgv_solve(tgv_domain* d, int32_t level, int32_t iterations, double* energy_gap_out)
{
    TgvNvtxRange nvtx_range_("tgv_solve");
    tgv_status st = check_domain(d);
    if (st != TGV_OK) return st;
    DeviceGuard g(d->device);
    TgvLevel* L;
    if ((st = get_level(d, level, &L)) != TGV_OK) return st;
    if (iterations < 0) return tgv_fail(d, TGV_ERR_INVALID_ARG, "iterations must be >= 0");
    if ((st = tgv_launch_iterations(d, *L, iterations)) != TGV_OK) return st;
    if (energy_gap_out) return tgv_launch_energy(d, *L, energy_gap_out);
    return TGV_OK;
}

tgv_status tgv_energy(tgv_domain* d, int32_t level, double* out)
{
    TgvNvtxRange nvtx_range_("tgv_energy");
    tgv_status st = check_domain(d);
    if (st != TGV_OK) return st;
    if (!out) return tgv_fail(d, TGV_ERR_INVALID_ARG, "null output");
    DeviceGuard g(d->device);
    TgvLevel* L;
    if ((st = get_level(d, level, &L)) != TGV_OK) return st;
    return tgv_launch_energy(d, *L, out);
}

tgv_status tgv_extract_field(tgv_domain* d, int32_t level, int32_t field, float* out, int64_t count)
{
    tgv_status st = check_domain(d);
    if (st != TGV_OK) return st;
    DeviceGuard g(d->device);
    TgvLevel* L;
    if ((st = get_level(d, level, &L)) != TGV_OK) return st;
    const int nc = ncomp_of(field);
    if (nc == 0) return tgv_fail(d, TGV_ERR_INVALID_ARG, "unknown field");
    const int64_t nvox = L->nb * TGV_BVOX;
    if (!out || count != nvox * nc) return tgv_fail(d, TGV_ERR_INVALID_ARG, "output size must be voxels * components");
    if (nvox == 0) return TGV_OK;
    const bool dev = is_device_ptr(out);
    float* dst = out;
    if (!dev) {
        if ((st = tgv_scratch(d, d->tmp, (size_t)count * 4)) != TGV_OK) return st;
        dst = (float*)d->tmp.ptr;
    }
    const void* f = field_ptr(*L, field);
    const bool fp32 = field == TGV_FIELD_U || field == TGV_FIELD_UBAR || d->prm.storage == TGV_STORAGE_FP32;
    const bool fx = d->prm.storage == TGV_STORAGE_FX16 && (field == TGV_FIELD_P || field == TGV_FIELD_Q);
    const DualScales ds = tgv_dual_scales(d->prm);
    const unsigned gr = grid1(count, 256, d->sm_count);
    if (fp32) field_extract_kernel<float><<<gr, 256, 0, d->stream>>>((const float*)f, dst, nvox, nc, 0.0f);
    else if (fx)
        field_extract_kernel<int16_t><<<gr, 256, 0, d->stream>>>((const int16_t*)f, dst, nvox, nc,
                                                                 field == TGV_FIELD_P ? ds.dsp : ds.dsq);
    else if (d->prm.storage == TGV_STORAGE_BF16)
        field_extract_kernel<__nv_bfloat16><<<gr, 256, 0, d->stream>>>((const __nv_bfloat16*)f, dst, nvox, nc, 0.0f);
    else field_extract_kernel<__half><<<gr, 256, 0, d->stream>>>((const __half*)f, dst, nvox, nc, 0.0f);
    d->launches++;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && !dev) e = cudaMemcpyAsync(out, dst, (size_t)count * 4, cudaMemcpyDeviceToHost, d->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    return tgv_cuda_check(d, e, "extract field");
}

tgv_status tgv_extract_mesh(tgv_domain* d, int32_t level, int64_t* nverts, int64_t* ntris)
{
    TgvNvtxRange nvtx_range_("tgv_extract_mesh");
    tgv_status st = check_domain(d);
    if (st != TGV_OK) return st;
    if (!nverts || !ntris) return tgv_fail(d, TGV_ERR_INVALID_ARG, "nverts and ntris must not be NULL");
    DeviceGuard g(d->device);
    TgvLevel* L;
    if ((st = get_level(d, level, &L)) != TGV_OK) return st;
    d->mesh_nv = d->mesh_nt = -1;
    return tgv_mesh_extract(d, *L, nverts, ntris);
}

tgv_status tgv_copy_mesh(tgv_domain* d, float* verts, int64_t nverts, int32_t* tris, int64_t ntris)
{
    tgv_status st = check_domain(d);
    if (st != TGV_OK) return st;
    if (d->mesh_nv < 0) return tgv_fail(d, TGV_ERR_STATE, "no mesh extracted");
    if (nverts != d->mesh_nv || ntris != d->mesh_nt || (nverts > 0 && !verts) || (ntris > 0 && !tris))
        return tgv_fail(d, TGV_ERR_INVALID_ARG, "counts must be those of the last tgv_extract_mesh");
    DeviceGuard g(d->device);
    cudaError_t e = cudaSuccess;
    if (nverts > 0) e = cudaMemcpyAsync(verts, d->mesh_v.ptr, (size_t)nverts * 12, cudaMemcpyDefault, d->stream);
    if (e == cudaSuccess && ntris > 0)
        e = cudaMemcpyAsync(tris, d->mesh_t.ptr, (size_t)ntris * 12, cudaMemcpyDefault, d->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    return tgv_cuda_check(d, e, "mesh copy");
}

tgv_status tgv_set_field(tgv_domain* d, int32_t level, int32_t field, const float* in, int64_t count)
{
    tgv_status st = check_domain(d);
    if (st != TGV_OK) return st;
    DeviceGuard g(d->device);
    TgvLevel* L;
    if ((st = get_level(d, level, &L)) != TGV_OK) return st;
    const int nc = ncomp_of(field);
    if (nc == 0) return tgv_fail(d, TGV_ERR_INVALID_ARG, "unknown field");
    const int64_t nvox = L->nb * TGV_BVOX;
    if (!in || count != nvox * nc) return tgv_fail(d, TGV_ERR_INVALID_ARG, "input size must be voxels * components");
    if (nvox == 0) return TGV_OK;
    const float* src = in;
    cudaError_t e = cudaSuccess;
    if (!is_device_ptr(in)) {
        if ((st = tgv_scratch(d, d->tmp, (size_t)count * 4)) != TGV_OK) return st;
        e = cudaMemcpyAsync(d->tmp.ptr, in, (size_t)count * 4, cudaMemcpyHostToDevice, d->stream);
        src = (const float*)d->tmp.ptr;
    }
    void* f = field_ptr(*L, field);
    const bool fp32 = field == TGV_FIELD_U || field == TGV_FIELD_UBAR || d->prm.storage == TGV_STORAGE_FP32;
    const bool fx = d->prm.storage == TGV_STORAGE_FX16 && (field == TGV_FIELD_P || field == TGV_FIELD_Q);
    const DualScales ds = tgv_dual_scales(d->prm);
    const unsigned gr = grid1(count, 256, d->sm_count);
    if (e == cudaSuccess) {
        if (fp32) field_set_kernel<float><<<gr, 256, 0, d->stream>>>((float*)f, src, nvox, nc, 0.0f);
        else if (fx)
            field_set_kernel<int16_t><<<gr, 256, 0, d->stream>>>((int16_t*)f, src, nvox, nc,
                                                                 field == TGV_FIELD_P ? ds.isp : ds.isq);
        else if (d->prm.storage == TGV_STORAGE_BF16)
            field_set_kernel<__nv_bfloat16><<<gr, 256, 0, d->stream>>>((__nv_bfloat16*)f, src, nvox, nc, 0.0f);
        else field_set_kernel<__half><<<gr, 256, 0, d->stream>>>((__half*)f, src, nvox, nc, 0.0f);
        d->launches++;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    return tgv_cuda_check(d, e, "set field");
}

tgv_status tgv_extract_histograms(tgv_domain* d, int32_t level, uint32_t* out, int64_t count)
{
    tgv_status st = check_domain(d);
    if (st != TGV_OK) return st;
    DeviceGuard g(d->device);
    TgvLevel* L;
    if ((st = get_level(d, level, &L)) != TGV_OK) return st;
    const int64_t nvox = L->nb * TGV_BVOX;
    if (!out || count != nvox * d->prm.nbins) return tgv_fail(d, TGV_ERR_INVALID_ARG, "output size must be voxels * nbins");
    if (nvox == 0) return TGV_OK;
    const bool dev = is_device_ptr(out);
    uint32_t* dst = out;
    if (!dev) {
        if ((st = tgv_scratch(d, d->tmp, (size_t)count * 4)) != TGV_OK) return st;
        dst = (uint32_t*)d->tmp.ptr;
    }
    hist_unpack_kernel<<<grid1(count, 256, d->sm_count), 256, 0, d->stream>>>(L->hist, dst, nvox, d->prm.nbins,
                                                                             (d->prm.nbins + 1) / 2);
    d->launches++;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && !dev) e = cudaMemcpyAsync(out, dst, (size_t)count * 4, cudaMemcpyDeviceToHost, d->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    return tgv_cuda_check(d, e, "extract histograms");
}

tgv_status tgv_set_histograms(tgv_domain* d, int32_t level, const uint32_t* in, int64_t count)
{
    tgv_status st = check_domain(d);
    if (st != TGV_OK) return st;
    DeviceGuard g(d->device);
    TgvLevel* L;
    if ((st = get_level(d, level, &L)) != TGV_OK) return st;
    const int64_t nvox = L->nb * TGV_BVOX;
    if (!in || count != nvox * d->prm.nbins) return tgv_fail(d, TGV_ERR_INVALID_ARG, "input size must be voxels * nbins");
    if (nvox == 0) return TGV_OK;
    const int npairs = (d->prm.nbins + 1) / 2;
    if ((st = tgv_scratch(d, d->tmp, (size_t)count * 4 + 256)) != TGV_OK) return st;
    unsigned int* maxc = (unsigned int*)((char*)d->tmp.ptr + (size_t)count * 4);
    const uint32_t* src = in;
    cudaError_t e = cudaMemsetAsync(maxc, 0, sizeof(unsigned int), d->stream);
    if (e == cudaSuccess && !is_device_ptr(in)) {
        e = cudaMemcpyAsync(d->tmp.ptr, in, (size_t)count * 4, cudaMemcpyHostToDevice, d->stream);
        src = (const uint32_t*)d->tmp.ptr;
    }
    if (e == cudaSuccess) {
        hist_pack_kernel<<<grid1(nvox * npairs, 256, d->sm_count), 256, 0, d->stream>>>(L->hist, src, nvox,
                                                                                      d->prm.nbins, npairs, maxc);
        d->launches++;
        e = cudaGetLastError();
    }
    unsigned int mx = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&mx, maxc, sizeof(mx), cudaMemcpyDeviceToHost, d->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    if ((st = tgv_cuda_check(d, e, "set histograms")) != TGV_OK) return st;
    if (mx > 65535) {
        cudaMemsetAsync(L->hist, 0, (size_t)npairs * nvox * 4, d->stream);
        L->max_votes = 0;
        return tgv_fail(d, TGV_ERR_BUDGET, "a histogram count exceeds 65535 (16-bit bins); histograms cleared");
    }
    L->max_votes = mx;
    return TGV_OK;
}

tgv_status tgv_reset(tgv_domain* d, int32_t level, int32_t clear_hist)
{
    TgvNvtxRange nvtx_range_("tgv_reset");
    tgv_status st = check_domain(d);
    if (st != TGV_OK) return st;
    DeviceGuard g(d->device);
    TgvLevel* L;
    if ((st = get_level(d, level, &L)) != TGV_OK) return st;
    const size_t vn = (size_t)L->nb * TGV_BVOX, sb = storage_bytes(d->prm.storage);
    cudaStream_t s = d->stream;
    cudaError_t e = cudaMemsetAsync(L->u, 0, vn * 4, s);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaMemsetAsync(L->ubar[k], 0, vn * 4, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(L->vbar[k], 0, 3 * vn * sb, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(L->p[k], 0, 3 * vn * sb, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(L->q[k], 0, 6 * vn * sb, s);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(L->v, 0, 3 * vn * sb, s);
    if (e == cudaSuccess && clear_hist) {
        e = cudaMemsetAsync(L->hist, 0, (size_t)((d->prm.nbins + 1) / 2) * vn * 4, s);
        L->max_votes = 0;
    }
    L->cur = 0;
    return tgv_cuda_check(d, e, "reset");
}

tgv_status tgv_prolong(tgv_domain* d, int32_t from_level)
{
    TgvNvtxRange nvtx_range_("tgv_prolong");
    tgv_status st = check_domain(d);
    if (st != TGV_OK) return st;
    DeviceGuard g(d->device);
    if (from_level < 0 || from_level + 1 >= (int32_t)d->levels.size())
        return tgv_fail(d, TGV_ERR_INVALID_ARG, "no finer level after from_level");
    TgvLevel& C = d->levels[from_level];
    TgvLevel& F = d->levels[from_level + 1];
    for (int a = 0; a < 3; ++a)
        if (C.origin[a] != F.origin[a]) return tgv_fail(d, TGV_ERR_INVALID_ARG, "levels must share the origin");
    if (fabs(F.h * 2.0 - C.h) > 1e-12 * C.h) return tgv_fail(d, TGV_ERR_INVALID_ARG, "fine h must be half the coarse h");
    const int64_t nfall = F.nb + F.nf;
    if (nfall == 0) return TGV_OK;
    std::unordered_map<uint64_t, int32_t> cidx;
    cidx.reserve((size_t)C.nb * 2);
    for (int64_t i = 0; i < C.nb; ++i)
        cidx.emplace(brick_key(C.coords[3 * i], C.coords[3 * i + 1], C.coords[3 * i + 2]), (int32_t)i);
    std::vector<int32_t> parent((size_t)nfall);
    auto fdiv2 = [](int32_t v) { return v >= 0 ? v / 2 : -((-v + 1) / 2); };
    for (int64_t i = 0; i < nfall; ++i) {
        auto it = cidx.find(
            brick_key(fdiv2(F.coords[3 * i]), fdiv2(F.coords[3 * i + 1]), fdiv2(F.coords[3 * i + 2])));
        parent[(size_t)i] = it == cidx.end() ? -1 : it->second;
    }
    if ((st = tgv_scratch(d, d->table, parent.size() * 4)) != TGV_OK) return st;
    cudaError_t e = cudaMemcpyAsync(d->table.ptr, parent.data(), parent.size() * 4, cudaMemcpyHostToDevice, d->stream);
    if (e == cudaSuccess) {
        const int o = 1 - F.cur;
        switch (d->prm.storage) {
        case TGV_STORAGE_FP32:
            prolong_kernel<float><<<(unsigned)nfall, TGV_BVOX, 0, d->stream>>>(
                C.u, (const float*)C.v, (const int32_t*)d->table.ptr, F.coords_dev, nfall, F.nb, F.u, F.ubar[F.cur],
                F.ubar[o], (float*)F.v, (float*)F.vbar[F.cur], (float*)F.vbar[o]);
            break;
        case TGV_STORAGE_BF16:
            prolong_kernel<__nv_bfloat16><<<(unsigned)nfall, TGV_BVOX, 0, d->stream>>>(
                C.u, (const __nv_bfloat16*)C.v, (const int32_t*)d->table.ptr, F.coords_dev, nfall, F.nb, F.u,
                F.ubar[F.cur], F.ubar[o], (__nv_bfloat16*)F.v, (__nv_bfloat16*)F.vbar[F.cur],
                (__nv_bfloat16*)F.vbar[o]);
            break;
        default:
            prolong_kernel<__half><<<(unsigned)nfall, TGV_BVOX, 0, d->stream>>>(
                C.u, (const __half*)C.v, (const int32_t*)d->table.ptr, F.coords_dev, nfall, F.nb, F.u, F.ubar[F.cur],
                F.ubar[o], (__half*)F.v, (__half*)F.vbar[F.cur], (__half*)F.vbar[o]);
        }
        d->launches++;
        e = cudaGetLastError();
    }
    const size_t vn = (size_t)F.nb * TGV_BVOX, sb = storage_bytes(d->prm.storage);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaMemsetAsync(F.p[k], 0, 3 * vn * sb, d->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(F.q[k], 0, 6 * vn * sb, d->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);  // `parent` is a host temporary
    return tgv_cuda_check(d, e, "prolong");
}

tgv_status tgv_set_work_list(tgv_domain* d, int32_t level, const int32_t* bricks, int64_t n)
{
    tgv_status st = check_domain(d);
    if (st != TGV_OK) return st;
    DeviceGuard g(d->device);
    TgvLevel* L;
    if ((st = get_level(d, level, &L)) != TGV_OK) return st;
    if (!bricks || n < 0) {  // back to every active brick
        L->work_gen++;
        if (L->work) {
            cudaError_t e = cudaStreamSynchronize(d->stream);  // queued launches may read the old list
            if (e != cudaSuccess) return tgv_cuda_check(d, e, "work list sync");
            cudaFree(L->work);
            d->bytes -= L->work_cap * 4;
        }
        L->work = nullptr;
        L->nwork = L->work_cap = 0;
        L->work_host.clear();
        return TGV_OK;
    }
    std::vector<int32_t> host((size_t)n);
    cudaError_t e = cudaMemcpy(host.data(), bricks, (size_t)n * 4, cudaMemcpyDefault);
    if (e != cudaSuccess) return tgv_cuda_check(d, e, "work list read");
    std::vector<uint8_t> seen((size_t)L->nb, 0);
    for (int32_t b : host) {
        if (b < 0 || b >= L->nb) return tgv_fail(d, TGV_ERR_INVALID_ARG, "work list entry is not an active brick");
        if (seen[(size_t)b]++) return tgv_fail(d, TGV_ERR_INVALID_ARG, "work list repeats a brick");
    }
    if (n > L->work_cap) {
        e = cudaStreamSynchronize(d->stream);
        if (e != cudaSuccess) return tgv_cuda_check(d, e, "work list sync");
        if (L->work) {
            cudaFree(L->work);
            d->bytes -= L->work_cap * 4;
            L->work = nullptr;
            L->work_cap = 0;
        }
        if ((st = dalloc(d, (void**)&L->work, (size_t)std::max<int64_t>(n, 1) * 4)) != TGV_OK) return st;
        L->work_cap = std::max<int64_t>(n, 1);
    }
    e = cudaMemcpyAsync(L->work, host.data(), (size_t)n * 4, cudaMemcpyHostToDevice, d->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);  // `host` is a temporary
    if (e != cudaSuccess) return tgv_cuda_check(d, e, "work list upload");
    L->nwork = n;
    L->work_gen++;
    L->work_host = std::move(host);
    return TGV_OK;
}

tgv_status tgv_solve_graph(tgv_domain* d, int32_t level, int32_t iterations, double* energy_gap_out)
{
    TgvNvtxRange nvtx_range_("tgv_solve_graph");
    tgv_status st = check_domain(d);
    if (st != TGV_OK) return st;
    DeviceGuard g(d->device);
    TgvLevel* L;
    if ((st = get_level(d, level, &L)) != TGV_OK) return st;
    if (iterations < 0) return tgv_fail(d, TGV_ERR_INVALID_ARG, "iterations must be >= 0");
    if (!d->stream) return tgv_fail(d, TGV_ERR_UNSUPPORTED, "graph capture needs a non-default stream");
    if (iterations > 0 && tgv_work_items(*L) > 0) {
        const int parity = L->cur;
        TgvLevel::Graph* hit = nullptr;
        for (auto& gr : L->graphs)
            if (gr.iters == iterations && gr.parity == parity && gr.gen == L->work_gen) hit = &gr;
        if (hit) {
            cudaError_t e = cudaGraphLaunch(hit->exec, d->stream);
            if (e != cudaSuccess) return tgv_cuda_check(d, e, "graph launch");
            d->launches += iterations;
            L->cur ^= iterations & 1;
        } else {
            // This call runs its iterations with plain launches (which also caches every
            // kernel's launch attributes); a graph of the same launches is captured for
            // the next call with the same count, starting parity and work list.
            if ((st = tgv_launch_iterations(d, *L, iterations)) != TGV_OK) return st;
            const int after = L->cur;
            const int64_t launches = d->launches;
            L->cur = parity;
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamBeginCapture(d->stream, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) {
                L->cur = after;
                return tgv_cuda_check(d, e, "begin capture");
            }
            st = tgv_launch_iterations(d, *L, iterations);
            e = cudaStreamEndCapture(d->stream, &graph);
            L->cur = after;  // capture recorded the launches without running them
            d->launches = launches;
            if (st != TGV_OK) return st;
            if (e != cudaSuccess) return tgv_cuda_check(d, e, "end capture");
            cudaGraphExec_t exec = nullptr;
            e = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return tgv_cuda_check(d, e, "graph instantiate");
            L->graphs.push_back({iterations, parity, L->work_gen, exec});
        }
    }
    if (energy_gap_out) return tgv_launch_energy(d, *L, energy_gap_out);
    return TGV_OK;
}

tgv_status tgv_synchronize(tgv_domain* d)
{
    tgv_status st = check_domain(d);
    if (st != TGV_OK) return st;
    DeviceGuard g(d->device);
    st = tgv_cuda_check(d, cudaStreamSynchronize(d->stream), "synchronize");
    if (st != TGV_OK) return st;
    return tgv_check_device_error(d);
}

int64_t tgv_domain_bytes(const tgv_domain* d) { return d ? d->bytes : 0; }

int64_t tgv_level_voxels(const tgv_domain* d, int32_t level)
{
    if (!d || level < 0 || level >= (int32_t)d->levels.size()) return 0;
    return d->levels[level].nb * TGV_BVOX;
}

int64_t tgv_launch_count(const tgv_domain* d) { return d ? d->launches : 0; }

}  // extern "C"
