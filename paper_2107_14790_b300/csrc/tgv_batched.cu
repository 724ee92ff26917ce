// Persistent batched solve of many independent chunks in one launch (Sec. 4.3: the
// treetop's parts are independent problems; Sec. 4.5: each is solved with its border
// cubes frozen).  The chunks are ranges of active bricks of one level with no link
// between them; chunk c runs its own number of iterations.
//
// Work is a sequence of tickets handed out by one global counter.  A ticket is one run
// of R consecutive bricks of one chunk in one iteration; tickets run iteration-major
// (iteration 0 of every chunk, then iteration 1 of every chunk that has one, ...), and
// within an iteration chunk by chunk.  A CTA takes a ticket, waits until every run of
// the chunk's previous iteration has completed (a per-chunk completion counter: the
// chunk's barrier between iterations, a bounded wait), sweeps the run's bricks with the
// paired machinery (tgv_pair_cta.cuh: bulk copies into shared memory, phase A duals,
// phase B primal step) and counts the run as completed.
//
// No CTA can wait forever on work that is not running: a CTA takes its next ticket only
// after finishing the previous one, tickets go out in increasing order, and a run only
// waits on runs of earlier iterations, whose tickets are smaller and were taken by CTAs
// that are running.  So progress never depends on which CTAs are resident; the waits
// are bounded all the same (tgv_params.wait_cycles; a CTA that gives up sets the error
// flag).
//
// Iteration k of a chunk reads ping-pong copy (cur + k) & 1 and writes the other; a chunk
// whose iteration count has the other parity than the largest one gets its ubar, vbar,
// p, q copied into the level's final copy afterwards, so the level keeps one current
// copy.
#include <string.h>

#include <algorithm>
#include <vector>

#include "tgv_pair_cta.cuh"
#include "tgv_nvtx.h"

template <typename S, typename D>
struct BatchArgs {
    PairArgs<S, D> pa;      // shared-memory layout, error flag, wait budget; pa.it reads copy
                            // cur (a chunk's even iterations; odd ones swap in and out)
    // segments of iterations with the same set of active chunks (chunks sorted by
    // iteration count, descending): segment j covers iterations [seg_k[j], seg_k[j+1])
    // with the first seg_a[j] chunks active, and tickets [seg_t[j], seg_t[j+1])
    const int64_t* seg_k;
    const int64_t* seg_t;
    const int32_t* seg_a;
    const int64_t* cum_runs;  // [nchunks + 1] runs per iteration of the chunks before c
    const int64_t* cfirst;    // [nchunks] first item of chunk c (sorted order)
    const int64_t* cend;      // [nchunks] one past its last item
    uint32_t* done;           // [nchunks] completed runs (zero at launch)
    unsigned long long* ticket;
    int32_t nseg, R;
    uint32_t off_task;        // shared-memory slot where thread 0 posts the CTA's task
};

namespace {

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// orders the generic-proxy writes this thread has observed before its later
// asynchronous-proxy (bulk copy) reads of global memory
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// largest index i in [0, n) with a[i] <= x (a ascending, a[0] <= x)
__device__ __forceinline__ int upper_index(const int64_t* a, int n, int64_t x)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

}  // namespace

template <typename S, typename D, int NB>
__global__ void __launch_bounds__(kThreads, 2) tgv_batched_kernel(const BatchArgs<S, D> B)
{
    extern __shared__ __align__(128) unsigned char smem[];
    int64_t* task = (int64_t*)(smem + B.off_task);  // first item, end item, chunk, parity, state
    const int t = threadIdx.x;
    uint64_t* bar = (uint64_t*)(smem + B.pa.off_bar);
    if (t == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init(&bar[2], 1);
        fence_mbar_init();
    }
    const int64_t total = B.seg_t[B.nseg];
    uint32_t parity = 0;
    for (;;) {
        if (t == 0) {
            int64_t state = 0;  // 0: no tickets left, 1: run, 2: a wait gave up
            const int64_t tk = (int64_t)atomicAdd(B.ticket, 1ull);
            if (tk < total) {
                const int j = upper_index(B.seg_t, B.nseg + 1, tk);
                const int64_t w = B.cum_runs[B.seg_a[j]];  // runs per iteration in segment j
                const int64_t k = B.seg_k[j] + (tk - B.seg_t[j]) / w;
                const int64_t r = (tk - B.seg_t[j]) % w;
                const int c = upper_index(B.cum_runs, B.seg_a[j] + 1, r);
                const int64_t nr = B.cum_runs[c + 1] - B.cum_runs[c];
                const int64_t i0 = B.cfirst[c] + (r - B.cum_runs[c]) * B.R;
                // the chunk's barrier: every run of its iteration k - 1 has completed (in the
                // test mode a count no run reaches, so the wait must run out)
                const uint32_t need = B.pa.wait_test ? 0xffffffffu : (uint32_t)(k * nr);
                state = 1;
                if (ld_acquire_u32(&B.done[c]) < need) {
                    const long long c0 = clock64();
                    for (;;) {
                        __nanosleep(128);
                        if (ld_acquire_u32(&B.done[c]) >= need) break;
                        if (clock64() - c0 > B.pa.wait_budget) {
                            state = 2;
                            break;
                        }
                    }
                }
                fence_proxy_async_global();
                task[0] = i0;
                task[1] = i0 + B.R < B.cend[c] ? i0 + B.R : B.cend[c];
                task[2] = c;
                task[3] = k & 1;
            }
            task[4] = state;
        }
        __syncthreads();
        const int64_t state = task[4];
        if (state != 1) {
            if (state == 2 && t == 0) atomicExch(B.pa.err, 1);
            break;
        }
        const uint32_t i0 = (uint32_t)task[0], i1 = (uint32_t)task[1];
        const int c = (int)task[2];
        PairCta<S, D, NB> C(B.pa, smem, task[3] != 0);
        if (!pair_sweep(C, OneRun{i1}, i0, parity, false)) break;
        __syncthreads();  // every store of the run has been issued
        if (t == 0) {
            __threadfence();
            atomicAdd(&B.done[c], 1u);
        }
    }
}

// Copies ubar, vbar, p, q of the listed bricks from the copy A reads to the copy A writes
// (chunks whose iteration count has the other parity than the largest one).
template <typename S, typename D>
__global__ void __launch_bounds__(256) batched_parity_copy_kernel(const int32_t* __restrict__ bricks,
                                                                 const IterArgs<S, D> A)
{
    const int64_t b = bricks[blockIdx.x];
    const int t = threadIdx.x;
    for (int i = t; i < TGV_BVOX; i += blockDim.x) A.ubar_out[b * TGV_BVOX + i] = A.ubar_in[b * TGV_BVOX + i];
    for (int i = t; i < 3 * TGV_BVOX; i += blockDim.x) {
        A.vbar_out[b * 3 * TGV_BVOX + i] = A.vbar_in[b * 3 * TGV_BVOX + i];
        A.p_out[b * 3 * TGV_BVOX + i] = A.p_in[b * 3 * TGV_BVOX + i];
    }
    for (int i = t; i < 6 * TGV_BVOX; i += blockDim.x) A.q_out[b * 6 * TGV_BVOX + i] = A.q_in[b * 6 * TGV_BVOX + i];
}

namespace {

// Host tables of one batched call (the device copy lives in the cache entry).
struct BatchPlan {
    std::vector<int64_t> seg_k, seg_t, cum_runs, cfirst, cend;
    std::vector<int32_t> seg_a, fix;  // fix: bricks needing the parity copy
    int64_t total = 0;
    int32_t maxit = 0;
};

// byte offsets of the tables in one device buffer (8-byte aligned)
struct BatchLayout {
    size_t ticket, done, seg_k, seg_t, seg_a, cum, cfirst, cend, fix, bytes, counters;
};

BatchLayout batch_layout(const BatchPlan& p, int nchunks)
{
    BatchLayout o;
    size_t off = 0;
    auto take = [&](size_t n) {
        const size_t at = off;
        off = (off + n + 15) / 16 * 16;
        return at;
    };
    o.ticket = take(8);
    o.done = take(4 * (size_t)nchunks);
    o.counters = off;  // ticket and done are zeroed before every launch
    o.seg_k = take(8 * p.seg_k.size());
    o.seg_t = take(8 * p.seg_t.size());
    o.seg_a = take(4 * p.seg_a.size());
    o.cum = take(8 * p.cum_runs.size());
    o.cfirst = take(8 * p.cfirst.size());
    o.cend = take(8 * p.cend.size());
    o.fix = take(4 * std::max<size_t>(1, p.fix.size()));
    o.bytes = off;
    return o;
}

uint64_t mix64(uint64_t h, uint64_t x)
{
    h ^= x + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
    return h;
}

template <typename S, typename D, int NB>
tgv_status launch_batched_t(tgv_domain* d, TgvLevel& L, const BatchPlan& plan, TgvLevel::Batch& E, int R)
{
    const uint32_t SB = sizeof(S), SD = sizeof(D);
    const int npairs = (d->prm.nbins + 1) / 2;
    const PairLayout LY = pair_layout(SB, SD, (uint32_t)npairs);
    const uint32_t tx = LY.tx, stage = LY.stage;
    uint32_t off = LY.end;
    BatchArgs<S, D> B;
    PairArgs<S, D>& P = B.pa;
    P.pn_bytes = LY.pn_bytes;
    P.off_pn = LY.off_pn;
    P.off_hal = LY.off_hal;
    P.off_nbr = LY.off_nbr;
    P.off_bar = LY.off_bar;
    off = (off + 15) / 16 * 16;
    B.off_task = off;
    off += 5 * 8;
    const size_t smem = off;
    auto kern = tgv_batched_kernel<S, D, NB>;
    int per_sm = 0;
    tgv_status st = tgv_kernel_setup((const void*)kern, kThreads, smem, &per_sm);
    if (st != TGV_OK) return tgv_fail(d, st, "batched kernel setup (shared memory attribute / occupancy) failed");
    if (per_sm < 1) return tgv_fail(d, TGV_ERR_UNSUPPORTED, "batched iteration kernel does not fit on an SM");
    int64_t grid = (int64_t)per_sm * d->sm_count;
    if (grid > plan.total) grid = plan.total;
    P.xrun = (uint32_t)R;
    P.err = d->err;
    P.wait_budget = tgv_wait_budget(d->prm);
    P.wait_test = d->prm.wait_test;
    P.stage_bytes = stage;
    P.tx_bytes = tx;
    const int cur0 = L.cur;
    P.it = tgv_make_iter_args<S, D>(d, L);
    P.it.work = nullptr;
    const BatchLayout lo = batch_layout(plan, (int)plan.cfirst.size());
    char* base = (char*)E.dev;
    B.seg_k = (const int64_t*)(base + lo.seg_k);
    B.seg_t = (const int64_t*)(base + lo.seg_t);
    B.seg_a = (const int32_t*)(base + lo.seg_a);
    B.cum_runs = (const int64_t*)(base + lo.cum);
    B.cfirst = (const int64_t*)(base + lo.cfirst);
    B.cend = (const int64_t*)(base + lo.cend);
    B.done = (uint32_t*)(base + lo.done);
    B.ticket = (unsigned long long*)(base + lo.ticket);
    B.nseg = (int32_t)plan.seg_a.size();
    B.R = R;
    cudaError_t e = cudaMemsetAsync(base, 0, lo.counters, d->stream);
    if (e == cudaSuccess && plan.total > 0) {
        kern<<<(unsigned)grid, kThreads, smem, d->stream>>>(B);
        d->launches++;
        e = cudaGetLastError();
    }
    const int fin = (cur0 + plan.maxit) & 1;  // the copy the level holds afterwards
    if (e == cudaSuccess && !plan.fix.empty()) {
        // the fixed chunks ended in copy fin ^ 1: copy it into fin
        L.cur = fin ^ 1;
        IterArgs<S, D> A = tgv_make_iter_args<S, D>(d, L);
        batched_parity_copy_kernel<S, D>
            <<<(unsigned)plan.fix.size(), 256, 0, d->stream>>>((const int32_t*)(base + lo.fix), A);
        d->launches++;
        e = cudaGetLastError();
    }
    L.cur = fin;
    return tgv_cuda_check(d, e, "batched kernel launch");
}

template <typename S, typename D = S>
tgv_status launch_batched_bins(tgv_domain* d, TgvLevel& L, const BatchPlan& p, TgvLevel::Batch& E, int R)
{
    switch (d->prm.nbins) {
    case 8: return launch_batched_t<S, D, 8>(d, L, p, E, R);
    case 10: return launch_batched_t<S, D, 10>(d, L, p, E, R);
    case 12: return launch_batched_t<S, D, 12>(d, L, p, E, R);
    default: return launch_batched_t<S, D, 0>(d, L, p, E, R);
    }
}

tgv_status launch_batched(tgv_domain* d, TgvLevel& L, const BatchPlan& p, TgvLevel::Batch& E, int R)
{
    switch (d->prm.storage) {
    case TGV_STORAGE_FP32: return launch_batched_bins<float>(d, L, p, E, R);
    case TGV_STORAGE_BF16: return launch_batched_bins<__nv_bfloat16>(d, L, p, E, R);
    case TGV_STORAGE_FP16: return launch_batched_bins<__half>(d, L, p, E, R);
    case TGV_STORAGE_FX16: return launch_batched_bins<__half, int16_t>(d, L, p, E, R);
    }
    return tgv_fail(d, TGV_ERR_INVALID_ARG, "unknown storage type");
}

}  // namespace

extern "C" TGV_API tgv_status tgv_solve_chunks(tgv_domain* d, int32_t level, int32_t nchunks, const int64_t* first,
                                               const int32_t* iterations, int32_t run_length)
{
    TgvNvtxRange nvtx_range_("tgv_solve_chunks");
    tgv_status st = tgv_check_domain(d);
    if (st != TGV_OK) return st;
    if (level < 0 || level >= (int32_t)d->levels.size()) return tgv_fail(d, TGV_ERR_INVALID_ARG, "level out of range");
    TgvLevel& L = d->levels[level];
    if (nchunks < 1 || !first || !iterations || run_length < 0 || run_length > 64)
        return tgv_fail(d, TGV_ERR_INVALID_ARG, "need nchunks >= 1, first[nchunks + 1], iterations[nchunks], run_length 0..64");
    if (L.work) return tgv_fail(d, TGV_ERR_INVALID_ARG, "batched solve with a work list set: clear it first");
    if (L.nb >= (int64_t)1 << 31) return tgv_fail(d, TGV_ERR_UNSUPPORTED, "batched solve of 2^31 bricks or more");
    for (int32_t c = 0; c < nchunks; ++c)
        if (first[c] < 0 || first[c + 1] <= first[c] || first[c + 1] > L.nb || iterations[c] < 0)
            return tgv_fail(d, TGV_ERR_INVALID_ARG, "chunks must be non-empty ascending brick ranges, iterations >= 0");
    // no link may join two chunks (each is an independent problem)
    if ((int64_t)L.nbr_host.size() < L.nb * TGV_NNBR) return tgv_fail(d, TGV_ERR_STATE, "neighbour rows missing");
    for (int32_t c = 0; c < nchunks; ++c)
        for (int64_t b = first[c]; b < first[c + 1]; ++b)
            for (int k = 0; k < TGV_NNBR; ++k) {
                const int32_t n = L.nbr_host[(size_t)b * TGV_NNBR + k];
                if (n >= 0 && n < L.nb && (n < first[c] || n >= first[c + 1]))
                    return tgv_fail(d, TGV_ERR_INVALID_ARG, "a link joins two chunks (chunk " + std::to_string(c) + ")");
            }
    // run length: 0 = 16 bricks (each run pays one pipeline start and one completion
    // count; the autotuner measures other lengths on the chunk mix it serves)
    const int R = run_length > 0 ? run_length : 16;
    // plan: chunks sorted by iteration count (descending, stable)
    std::vector<int32_t> ord(nchunks);
    for (int32_t c = 0; c < nchunks; ++c) ord[c] = c;
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) { return iterations[a] > iterations[b]; });
    BatchPlan p;
    p.maxit = iterations[ord[0]];
    p.cum_runs.push_back(0);
    for (int32_t c : ord) {
        const int64_t len = first[c + 1] - first[c];
        const int64_t nr = (len + R - 1) / R;
        if ((int64_t)iterations[c] * nr >= (int64_t)1 << 31)
            return tgv_fail(d, TGV_ERR_UNSUPPORTED, "iterations x runs of a chunk must stay below 2^31");
        p.cfirst.push_back(first[c]);
        p.cend.push_back(first[c + 1]);
        p.cum_runs.push_back(p.cum_runs.back() + nr);
    }
    // segments between distinct iteration counts
    int64_t tk = 0, k0 = 0;
    for (int32_t a = nchunks; a >= 1; --a) {
        // chunks [0, a) are active for iterations [k0, iterations of chunk a-1)
        const int64_t k1 = iterations[ord[a - 1]];
        if (k1 > k0) {
            p.seg_k.push_back(k0);
            p.seg_t.push_back(tk);
            p.seg_a.push_back(a);
            tk += (k1 - k0) * p.cum_runs[a];
            k0 = k1;
        }
    }
    p.seg_k.push_back(k0);
    p.seg_t.push_back(tk);
    p.total = tk;
    if (p.seg_a.empty()) p.seg_a.push_back(1);  // no iterations at all: the kernel sees total = 0
    for (int32_t c = 0; c < nchunks; ++c)
        if (((p.maxit - iterations[c]) & 1) != 0)
            for (int64_t b = first[c]; b < first[c + 1]; ++b) p.fix.push_back((int32_t)b);
    // the cache entry for this plan (device tables, and a CUDA graph of the call)
    uint64_t key = mix64(0x243f6a8885a308d3ull, (uint64_t)R);
    key = mix64(key, (uint64_t)L.cur);
    key = mix64(key, (uint64_t)nchunks);
    for (int32_t c = 0; c <= nchunks; ++c) key = mix64(key, (uint64_t)first[c]);
    for (int32_t c = 0; c < nchunks; ++c) key = mix64(key, (uint64_t)(uint32_t)iterations[c]);
    DeviceGuard g(d->device);
    TgvLevel::Batch* E = nullptr;
    for (auto& x : L.batches)
        if (x.key == key) E = &x;
    if (!E) {
        const BatchLayout lo = batch_layout(p, nchunks);
        std::vector<char> host(lo.bytes, 0);
        auto put = [&](size_t at, const void* src, size_t n) {
            if (n) memcpy(host.data() + at, src, n);
        };
        put(lo.seg_k, p.seg_k.data(), 8 * p.seg_k.size());
        put(lo.seg_t, p.seg_t.data(), 8 * p.seg_t.size());
        put(lo.seg_a, p.seg_a.data(), 4 * p.seg_a.size());
        put(lo.cum, p.cum_runs.data(), 8 * p.cum_runs.size());
        put(lo.cfirst, p.cfirst.data(), 8 * p.cfirst.size());
        put(lo.cend, p.cend.data(), 8 * p.cend.size());
        put(lo.fix, p.fix.data(), 4 * p.fix.size());
        TgvLevel::Batch nb;
        nb.key = key;
        if (cudaMalloc(&nb.dev, lo.bytes) != cudaSuccess) {
            cudaGetLastError();
            return tgv_fail(d, TGV_ERR_OUT_OF_MEMORY, "batched solve tables");
        }
        d->bytes += (int64_t)lo.bytes;
        nb.bytes = lo.bytes;
        cudaError_t e = cudaMemcpyAsync(nb.dev, host.data(), lo.bytes, cudaMemcpyHostToDevice, d->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
        if (e != cudaSuccess) {
            cudaFree(nb.dev);
            return tgv_cuda_check(d, e, "batched solve tables upload");
        }
        if (L.batches.size() >= 16) {  // keep the cache small: drop the oldest entry
            if (L.batches.front().exec) cudaGraphExecDestroy(L.batches.front().exec);
            cudaFree(L.batches.front().dev);
            d->bytes -= (int64_t)L.batches.front().bytes;
            L.batches.erase(L.batches.begin());
        }
        L.batches.push_back(nb);
        E = &L.batches.back();
    }
    if (E->exec) {
        d->launches += E->launches;
        L.cur = (L.cur + p.maxit) & 1;
        return tgv_cuda_check(d, cudaGraphLaunch(E->exec, d->stream), "batched graph launch");
    }
    if (!d->stream) return launch_batched(d, L, p, *E, R);
    // first call with this plan on a stream: capture the call into a graph, then launch it
    const int cur0 = L.cur;
    const int64_t l0 = d->launches;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(d->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return tgv_cuda_check(d, e, "begin capture");
    st = launch_batched(d, L, p, *E, R);
    e = cudaStreamEndCapture(d->stream, &graph);
    if (st != TGV_OK) {
        if (graph) cudaGraphDestroy(graph);
        L.cur = cur0;
        return st;
    }
    if (e != cudaSuccess) return tgv_cuda_check(d, e, "end capture");
    e = cudaGraphInstantiate(&E->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return tgv_cuda_check(d, e, "graph instantiate");
    E->launches = d->launches - l0;
    return tgv_cuda_check(d, cudaGraphLaunch(E->exec, d->stream), "batched graph launch");
}
