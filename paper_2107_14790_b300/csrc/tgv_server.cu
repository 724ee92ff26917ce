// Serving engine: chunk-solve requests share the fused iteration launches
// (continuous batching).
//
// The paper splits the domain into independent treetop-leaf parts whose
// border cubes (set B) are frozen (Sec. 4.3, Sec. 4.5); every part is an
// independent problem.  Here a request is one such part (active bricks, a
// frozen shell, histograms, an iteration count).  All requests of a server
// live in one arena level of fixed capacity (the HBM budget): active bricks in
// [0, cap_active), frozen bricks in [cap_active, cap_active + cap_frozen), each
// request in one contiguous range of each region.  Neighbour links never
// leave a request, so one launch of the fused kernel over the work list of
// all running requests advances each of them by one iteration exactly as a
// launch over that request alone would.
//
// submit() admits a request if both ranges fit (TGV_ERR_BUDGET otherwise: the
// caller keeps it queued), step() queues iterations for every running
// request up to the next completion, extract() copies a finished request's u
// out and releases its ranges.  Host inputs go through a pinned staging ring
// so that nothing on the request path synchronises the device.
#include <string.h>

#include <algorithm>
#include <map>
#include <unordered_map>
#include <vector>

#include "tgv_internal.cuh"
#include "tgv_nvtx.h"

namespace {

// First-fit allocator of index ranges [0, cap).
class RangeAlloc {
public:
    void init(int64_t cap)
    {
        free_.clear();
        if (cap > 0) free_[0] = cap;
        cap_ = cap;
    }
    bool alloc(int64_t n, int64_t* off)
    {
        if (n == 0) {
            *off = 0;
            return true;
        }
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const int64_t rem = it->second - n, o = it->first;
                free_.erase(it);
                if (rem) free_[o + n] = rem;
                return true;
            }
        }
        return false;
    }
    void release(int64_t off, int64_t n)
    {
        if (n == 0) return;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + n == next->first) {
            n += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += n;
                return;
            }
        }
        free_[off] = n;
    }
    int64_t free_total() const
    {
        int64_t s = 0;
        for (auto& kv : free_) s += kv.second;
        return s;
    }

private:
    std::map<int64_t, int64_t> free_;
    int64_t cap_ = 0;
};

struct Request {
    int64_t a0 = 0, nb = 0;  // active range
    int64_t f0 = 0, nf = 0;  // frozen range (offset inside the frozen region)
    int32_t remaining = 0;
    int32_t iterations = 0;
    bool done = false;
};

// Pinned host staging ring: each use waits for the copy that last used its bytes.
class StagingRing {
public:
    tgv_status init(size_t bytes)
    {
        if (cudaHostAlloc(&base_, bytes, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            base_ = nullptr;
            return TGV_ERR_OUT_OF_MEMORY;
        }
        cap_ = bytes;
        return TGV_OK;
    }
    void destroy()
    {
        for (auto& p : pending_) cudaEventDestroy(p.ev);
        pending_.clear();
        if (base_) cudaFreeHost(base_);
        base_ = nullptr;
    }
    size_t capacity() const { return cap_; }
    // returns a host pointer to `bytes` bytes, or nullptr if larger than the ring
    char* get(size_t bytes)
    {
        bytes = (bytes + 255) / 256 * 256;
        if (bytes > cap_) return nullptr;
        if (head_ + bytes > cap_) head_ = 0;
        const size_t lo = head_, hi = head_ + bytes;
        // wait for earlier copies whose source bytes overlap [lo, hi)
        for (auto it = pending_.begin(); it != pending_.end();) {
            if (it->lo < hi && lo < it->hi) {
                cudaEventSynchronize(it->ev);
                cudaEventDestroy(it->ev);
                it = pending_.erase(it);
            } else {
                ++it;
            }
        }
        head_ = hi;
        last_lo_ = lo;
        last_hi_ = hi;
        return base_ + lo;
    }
    // marks the bytes of the last get() busy until the stream reaches this point
    void busy_until(cudaStream_t s)
    {
        cudaEvent_t ev;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            cudaStreamSynchronize(s);
            return;
        }
        cudaEventRecord(ev, s);
        pending_.push_back({last_lo_, last_hi_, ev});
    }

private:
    struct Pending {
        size_t lo, hi;
        cudaEvent_t ev;
    };
    char* base_ = nullptr;
    size_t cap_ = 0, head_ = 0, last_lo_ = 0, last_hi_ = 0;
    std::vector<Pending> pending_;
};

inline uint64_t key3(int32_t x, int32_t y, int32_t z)
{
    const uint64_t B = (uint64_t)1 << 20;
    return (((uint64_t)(z + (int64_t)B) * (2 * B)) + (uint64_t)(y + (int64_t)B)) * (2 * B) + (uint64_t)(x + (int64_t)B);
}

const int kOffsets[TGV_NNBR][3] = {
    {+1, 0, 0}, {-1, 0, 0}, {0, +1, 0}, {0, -1, 0}, {0, 0, +1}, {0, 0, -1},
    {-1, +1, 0}, {-1, 0, +1}, {+1, -1, 0}, {0, -1, +1}, {+1, 0, -1}, {0, +1, -1}};

bool device_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

struct tgv_server {
    tgv_domain* dom = nullptr;
    cudaStream_t copy_stream = nullptr;
    int64_t cap_active = 0, cap_frozen = 0;
    RangeAlloc act, frz;
    std::unordered_map<uint64_t, Request> reqs;
    uint64_t next_ticket = 1;
    bool work_dirty = true;
    int64_t running = 0;
    StagingRing ring;
    unsigned int* maxc = nullptr;  // device word for the histogram range check
    int64_t iterations_run = 0;
    int64_t voxel_updates = 0;
};

extern "C" {

tgv_status tgv_server_create(const tgv_server_cfg* cfg, const tgv_params* prm, void* stream, tgv_server** out)
{
    if (!out) return TGV_ERR_INVALID_ARG;
    *out = nullptr;
    if (!cfg || !prm || !stream) return TGV_ERR_INVALID_ARG;
    if (cfg->capacity_bricks <= 0 || cfg->capacity_frozen < 0) return TGV_ERR_INVALID_ARG;
    if (prm->nbins < 2 || prm->nbins > TGV_MAX_BINS) return TGV_ERR_INVALID_ARG;
    if (prm->storage < TGV_STORAGE_FP32 || prm->storage > TGV_STORAGE_FX16) return TGV_ERR_INVALID_ARG;
    if (prm->x_run < 0 || prm->x_run > 64) return TGV_ERR_INVALID_ARG;
    if (prm->hist_form != TGV_HIST_GATHER && prm->hist_form != TGV_HIST_SCATTER) return TGV_ERR_INVALID_ARG;
    tgv_server* s = new (std::nothrow) tgv_server();
    if (!s) return TGV_ERR_OUT_OF_MEMORY;
    s->cap_active = cfg->capacity_bricks;
    s->cap_frozen = cfg->capacity_frozen;
    tgv_status st = tgv_create_arena(prm, (cudaStream_t)stream, s->cap_active, s->cap_frozen, &s->dom);
    if (st == TGV_OK) st = s->ring.init(cfg->staging_bytes > 0 ? (size_t)cfg->staging_bytes : (size_t)256 << 20);
    if (st == TGV_OK && cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
        st = TGV_ERR_CUDA;
    if (st == TGV_OK && cudaMalloc(&s->maxc, sizeof(unsigned int)) != cudaSuccess) st = TGV_ERR_OUT_OF_MEMORY;
    if (st != TGV_OK) {
        cudaGetLastError();
        tgv_server_destroy(s);
        return st;
    }
    s->act.init(s->cap_active);
    s->frz.init(s->cap_frozen);
    *out = s;
    return TGV_OK;
}

void tgv_server_destroy(tgv_server* s)
{
    if (!s) return;
    if (s->dom) {
        cudaStreamSynchronize(s->dom->stream);
        tgv_destroy_domain(s->dom);
    }
    if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
    if (s->maxc) cudaFree(s->maxc);
    s->ring.destroy();
    cudaGetLastError();
    delete s;
}

tgv_status tgv_server_submit(tgv_server* s, const tgv_level_desc* chunk, const uint32_t* hist, int32_t iterations,
                             uint64_t* ticket)
{
    if (!s || !chunk || !hist || !ticket || iterations < 0) return TGV_ERR_INVALID_ARG;
    tgv_domain* d = s->dom;
    if (d->broken) return TGV_ERR_STATE;
    const int64_t nb = chunk->nbricks, nf = chunk->nfrozen;
    if (nb <= 0 || nf < 0 || !chunk->brick_coords || (nf > 0 && !chunk->frozen_coords)) return TGV_ERR_INVALID_ARG;
    if (nb > s->cap_active || nf > s->cap_frozen) return TGV_ERR_INVALID_ARG;  // can never fit
    // neighbour rows of the request's active bricks, in arena indices
    std::unordered_map<uint64_t, int64_t> index;
    index.reserve((size_t)(nb + nf) * 2);
    for (int64_t i = 0; i < nb + nf; ++i) {
        const int32_t* c = i < nb ? chunk->brick_coords + 3 * i : chunk->frozen_coords + 3 * (i - nb);
        for (int a = 0; a < 3; ++a)
            if (c[a] < -(1 << 19) || c[a] >= (1 << 19)) return TGV_ERR_INVALID_ARG;
        if (!index.emplace(key3(c[0], c[1], c[2]), i).second) return TGV_ERR_INVALID_ARG;
    }
    {
        // every host input is staged through the pinned ring in one piece
        const size_t need_rows = (size_t)nb * TGV_NNBR * 4, need_fv = 3 * (size_t)nf * TGV_BVOX * 4;
        const size_t need_hist = device_ptr(hist) ? 0 : (size_t)nb * TGV_BVOX * d->prm.nbins * 4;
        if (std::max(std::max(need_rows, need_fv), need_hist) > s->ring.capacity())
            return tgv_fail(d, TGV_ERR_INVALID_ARG, "a host input is larger than the staging ring (staging_bytes)");
    }
    Request r;
    if (!s->act.alloc(nb, &r.a0)) return TGV_ERR_BUDGET;
    if (!s->frz.alloc(nf, &r.f0)) {
        s->act.release(r.a0, nb);
        return TGV_ERR_BUDGET;
    }
    r.nb = nb;
    r.nf = nf;
    r.remaining = r.iterations = iterations;
    r.done = iterations == 0;
    TgvLevel& L = d->levels[0];
    cudaStream_t st = d->stream;
    const size_t sb = storage_bytes(d->prm.storage);
    const int npairs = (d->prm.nbins + 1) / 2;
    const int64_t nvox = nb * TGV_BVOX;
    cudaError_t e = cudaSuccess;
    // 1. neighbour rows
    {
        int32_t* rows = (int32_t*)s->ring.get((size_t)nb * TGV_NNBR * 4);
        if (!rows) e = cudaErrorMemoryAllocation;
        for (int64_t i = 0; e == cudaSuccess && i < nb; ++i) {
            const int32_t* c = chunk->brick_coords + 3 * i;
            for (int k = 0; k < TGV_NNBR; ++k) {
                auto it = index.find(key3(c[0] + kOffsets[k][0], c[1] + kOffsets[k][1], c[2] + kOffsets[k][2]));
                int32_t v = -1;
                if (it != index.end()) v = (int32_t)(it->second < nb ? r.a0 + it->second : s->cap_active + r.f0 + (it->second - nb));
                rows[i * TGV_NNBR + k] = v;
            }
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(L.nbr + r.a0 * TGV_NNBR, rows, (size_t)nb * TGV_NNBR * 4,
                                                  cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) std::copy(rows, rows + nb * TGV_NNBR, L.nbr_host.begin() + r.a0 * TGV_NNBR);
        if (e == cudaSuccess) s->ring.busy_until(st);
    }
    // 2. active state: zero in both ping-pong copies
    {
        const size_t o = (size_t)r.a0 * TGV_BVOX, n = (size_t)nvox;
        if (e == cudaSuccess) e = cudaMemsetAsync(L.u + o, 0, n * 4, st);
        for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
            e = cudaMemsetAsync(L.ubar[k] + o, 0, n * 4, st);
            if (e == cudaSuccess) e = cudaMemsetAsync((char*)L.vbar[k] + 3 * o * sb, 0, 3 * n * sb, st);
            if (e == cudaSuccess) e = cudaMemsetAsync((char*)L.p[k] + 3 * o * sb, 0, 3 * n * sb, st);
            if (e == cudaSuccess) e = cudaMemsetAsync((char*)L.q[k] + 6 * o * sb, 0, 6 * n * sb, st);
        }
        if (e == cudaSuccess) e = cudaMemsetAsync((char*)L.v + 3 * o * sb, 0, 3 * n * sb, st);
    }
    // 3. frozen shell: u and v constants in both copies (zero where not given)
    if (nf > 0 && e == cudaSuccess) {
        const size_t fo = (size_t)(s->cap_active + r.f0) * TGV_BVOX, n = (size_t)nf * TGV_BVOX;
        float* u_dst[3] = {L.u, L.ubar[0], L.ubar[1]};
        void* v_dst[3] = {L.v, L.vbar[0], L.vbar[1]};
        if (chunk->frozen_u) {
            float* hb = (float*)s->ring.get(n * 4);
            if (!hb) e = cudaErrorMemoryAllocation;
            else {
                memcpy(hb, chunk->frozen_u, n * 4);
                for (int k = 0; k < 3 && e == cudaSuccess; ++k)
                    e = cudaMemcpyAsync(u_dst[k] + fo, hb, n * 4, cudaMemcpyHostToDevice, st);
                s->ring.busy_until(st);
            }
        } else {
            for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaMemsetAsync(u_dst[k] + fo, 0, n * 4, st);
        }
        if (e == cudaSuccess && chunk->frozen_v) {
            float* hb = (float*)s->ring.get(3 * n * 4);
            tgv_status ts = tgv_scratch(d, d->tmp, 3 * n * 4 + (size_t)nvox * d->prm.nbins * 4);
            if (!hb || ts != TGV_OK) e = cudaErrorMemoryAllocation;
            else {
                memcpy(hb, chunk->frozen_v, 3 * n * 4);
                e = cudaMemcpyAsync(d->tmp.ptr, hb, 3 * n * 4, cudaMemcpyHostToDevice, st);
                s->ring.busy_until(st);
                for (int k = 0; k < 3 && e == cudaSuccess; ++k)
                    tgv_launch_f32_to_storage(d, (const float*)d->tmp.ptr, (char*)v_dst[k] + 3 * fo * sb, 3 * (int64_t)n);
            }
        } else if (e == cudaSuccess) {
            for (int k = 0; k < 3 && e == cudaSuccess; ++k)
                e = cudaMemsetAsync((char*)v_dst[k] + 3 * fo * sb, 0, 3 * n * sb, st);
        }
    }
    // 4. histograms (host or device [voxel][nbins] uint32), packed into the request's range
    if (e == cudaSuccess) {
        const uint32_t* src = hist;
        const size_t hbytes = (size_t)nvox * d->prm.nbins * 4;
        if (!device_ptr(hist)) {
            tgv_status ts = tgv_scratch(d, d->tmp, hbytes + 3 * (size_t)nf * TGV_BVOX * 4);
            char* hb = ts == TGV_OK ? s->ring.get(hbytes) : nullptr;
            if (!hb) e = cudaErrorMemoryAllocation;
            else {
                uint32_t mx = 0;
                const size_t cnt = hbytes / 4;
                for (size_t i = 0; i < cnt; ++i) {
                    const uint32_t v = hist[i];
                    ((uint32_t*)hb)[i] = v;
                    mx = v > mx ? v : mx;
                }
                if (mx > 65535) {
                    s->act.release(r.a0, nb);
                    s->frz.release(r.f0, nf);
                    return tgv_fail(d, TGV_ERR_INVALID_ARG, "a histogram count exceeds 65535");
                }
                char* dst = (char*)d->tmp.ptr + 3 * (size_t)nf * TGV_BVOX * 4;  // after the frozen-v staging
                e = cudaMemcpyAsync(dst, hb, hbytes, cudaMemcpyHostToDevice, st);
                s->ring.busy_until(st);
                src = (const uint32_t*)dst;
            }
        }
        if (e == cudaSuccess) e = cudaMemsetAsync(s->maxc, 0, sizeof(unsigned int), st);
        if (e == cudaSuccess) {
            tgv_launch_hist_pack(d, L.hist + (size_t)r.a0 * npairs * TGV_BVOX, src, nvox, s->maxc);
            e = cudaGetLastError();
        }
    }
    if (e != cudaSuccess) {
        s->act.release(r.a0, nb);
        s->frz.release(r.f0, nf);
        return tgv_cuda_check(d, e, "request admission");
    }
    *ticket = s->next_ticket++;
    s->reqs[*ticket] = r;
    if (!r.done) {
        s->running++;
        s->work_dirty = true;
    }
    return TGV_OK;
}

tgv_status tgv_server_step(tgv_server* s, int32_t max_iterations, int32_t* finished)
{
    TgvNvtxRange nvtx_range_("tgv_server_step");
    if (!s || max_iterations < 0) return TGV_ERR_INVALID_ARG;
    tgv_domain* d = s->dom;
    if (d->broken) return TGV_ERR_STATE;
    if (finished) *finished = 0;
    if (s->running == 0 || max_iterations == 0) return TGV_OK;
    TgvLevel& L = d->levels[0];
    int32_t k = max_iterations;
    for (auto& kv : s->reqs)
        if (!kv.second.done) k = std::min(k, kv.second.remaining);
    if (s->work_dirty) {
        int64_t n = 0;
        for (auto& kv : s->reqs)
            if (!kv.second.done) n += kv.second.nb;
        int32_t* w = (int32_t*)s->ring.get((size_t)n * 4);
        if (!w) return tgv_fail(d, TGV_ERR_BUDGET, "work list larger than the staging ring");
        int64_t o = 0;
        for (auto& kv : s->reqs)
            if (!kv.second.done)
                for (int64_t i = 0; i < kv.second.nb; ++i) w[o++] = (int32_t)(kv.second.a0 + i);
        if (n > L.work_cap) {
            cudaError_t e = cudaStreamSynchronize(d->stream);
            if (e != cudaSuccess) return tgv_cuda_check(d, e, "work list sync");
            if (L.work) cudaFree(L.work);
            L.work = nullptr;
            const int64_t cap = std::max<int64_t>(n, s->cap_active);
            e = cudaMalloc(&L.work, (size_t)cap * 4);
            if (e != cudaSuccess) {
                cudaGetLastError();
                L.work_cap = 0;
                return tgv_fail(d, TGV_ERR_OUT_OF_MEMORY, "work list allocation failed");
            }
            L.work_cap = cap;
        }
        cudaError_t e = cudaMemcpyAsync(L.work, w, (size_t)n * 4, cudaMemcpyHostToDevice, d->stream);
        if (e != cudaSuccess) return tgv_cuda_check(d, e, "work list upload");
        s->ring.busy_until(d->stream);
        L.nwork = n;
        L.work_gen++;
        L.work_host.assign(w, w + n);
        s->work_dirty = false;
    }
    tgv_status st = tgv_launch_iterations(d, L, k);
    if (st != TGV_OK) return st;
    s->iterations_run += k;
    s->voxel_updates += L.nwork * TGV_BVOX * (int64_t)k;
    int32_t fin = 0;
    for (auto& kv : s->reqs) {
        Request& r = kv.second;
        if (r.done) continue;
        r.remaining -= k;
        if (r.remaining == 0) {
            r.done = true;
            s->running--;
            s->work_dirty = true;
            fin++;
        }
    }
    if (finished) *finished = fin;
    return TGV_OK;
}

tgv_status tgv_server_poll(tgv_server* s, uint64_t ticket, int32_t* done)
{
    if (!s || !done) return TGV_ERR_INVALID_ARG;
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return TGV_ERR_INVALID_ARG;
    *done = it->second.done ? 1 : 0;
    return TGV_OK;
}

tgv_status tgv_server_extract(tgv_server* s, uint64_t ticket, float* u_out, int64_t count)
{
    if (!s || !u_out) return TGV_ERR_INVALID_ARG;
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return TGV_ERR_INVALID_ARG;
    Request& r = it->second;
    if (!r.done) return tgv_fail(s->dom, TGV_ERR_STATE, "request still running");
    if (count != r.nb * TGV_BVOX) return TGV_ERR_INVALID_ARG;
    tgv_domain* d = s->dom;
    // u is updated in place, so after the request's last queued iteration its range is final
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev, d->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->copy_stream, ev, 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(u_out, d->levels[0].u + (size_t)r.a0 * TGV_BVOX, (size_t)count * 4, cudaMemcpyDefault,
                            s->copy_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->copy_stream);
    cudaEventDestroy(ev);
    if (e != cudaSuccess) return tgv_cuda_check(d, e, "extract");
    s->act.release(r.a0, r.nb);
    s->frz.release(r.f0, r.nf);
    s->reqs.erase(it);
    return TGV_OK;
}

int64_t tgv_server_free_bricks(const tgv_server* s) { return s ? s->act.free_total() : 0; }

const char* tgv_server_last_error(const tgv_server* s) { return s && s->dom ? s->dom->last_error.c_str() : "null server"; }

int64_t tgv_server_running(const tgv_server* s) { return s ? s->running : 0; }

int64_t tgv_server_voxel_updates(const tgv_server* s) { return s ? s->voxel_updates : 0; }

tgv_status tgv_server_synchronize(tgv_server* s)
{
    if (!s) return TGV_ERR_INVALID_ARG;
    return tgv_synchronize(s->dom);
}

}  // extern "C"
