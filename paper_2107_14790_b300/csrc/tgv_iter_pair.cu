// Pipelined, paired form of the fused TGV primal-dual iteration (the
// arithmetic of tgv_iter_kernel in tgv_solve.cu: Eq. 2-3, Sec. 3.2).
//
// Persistent CTAs; each of threads 0-255 owns the x-adjacent voxel pair
// (2j, 2j+1) of one row of the brick in hand, so shared-memory and global
// accesses are 64-bit (two FP32 or two 16-bit values) and the x-neighbour
// inside the pair comes from registers.  FP32 duals add four halo warps
// (384 threads) that compute the halo duals; 16-bit duals run 256 threads
// that do both.  Each brick's whole state -- u, ubar,
// v, vbar, p, q and the packed histogram, contiguous per brick -- arrives in
// shared memory through seven cp.async.bulk copies completed on an mbarrier,
// double-buffered: while one brick is computed, the next is in flight.
//
// Work items are taken in runs of R consecutive items (run r by CTA r mod
// grid).  Consecutive items of a run are usually x-neighbouring bricks, and
// then the two x-face halos pass between them on chip instead of being
// recomputed from scattered (stride-8) global loads:
//   * the new p_x on the x = 7 layer of brick i is what brick i+1 needs on its
//     -x face: phase A of brick i writes it straight into brick i+1's halo slot;
//   * brick i needs the new q on the x = 0 layer of brick i+1, which only
//     phase A of brick i+1 produces, after phase B of brick i: the v update of
//     brick i's x = 7 voxels leaves the +x term out (it is added last), parks
//     the partial sum, and phase A of brick i+1 completes it and stores the
//     x = 6, 7 pair (the x = 6 results wait in brick i's dead v and vbar slots,
//     so no row is written in two pieces).
// Phase B of one brick and phase A of the next touch different stages except
// for these hand-over slots, which only lanes of one warp share: a warp goes from
// one to the other after a warp sync, and one CTA barrier closes each interval.
// The dual updates use explicitly rounded arithmetic, so a dual recomputed as
// a halo equals the owner's bit for bit and results do not depend on R, the
// grid size or the order of the work items.
//
// The other halo duals (new p on the -y/-z face layers, new q on the +y/+z
// layers, and the x faces when the neighbour is not the adjacent item) are
// recomputed here in warp-uniform tasks (single voxels on the x faces, pairs on
// the y and z faces): with 256 threads the 384 halo voxels split into exactly one
// task per thread; the four halo warps of the FP32 form take one y/z face each
// and half an x face when it is not handed over.  Task inputs are loaded into
// registers before the CTA waits for its stage.
//
// The bin count is a template parameter for 8, 10 and 12 bins (0 = read at
// run time).  Every mbarrier wait is bounded (tgv_params.wait_cycles, about a
// second by default); a CTA that gives up sets the domain's error flag, waits
// (bounded, default budget) for its copies in flight and returns.
#include <math.h>

#include <vector>
#include "tgv_pair_cta.cuh"

// FP32 duals: 384 threads, the halo duals on four warps of their own (two CTAs per SM, as
// the two 45 KB stages allow); 16-bit duals: 256 threads with the halo tasks spread over
// the owners of the pairs (three CTAs per SM at 80 registers)
template <typename D> constexpr bool kPairHaloWarps = sizeof(D) == 4;
template <typename D> constexpr int kPairThreads = PairCta<float, D, 0, kPairHaloWarps<D>>::kCtaThreads;

// The level kernel: CTA r takes runs r, r + G, r + 2G, ... of R consecutive work items
// (G = grid size) and sweeps them with the paired machinery.
template <typename S, typename D, int NB>
__global__ void __launch_bounds__(kPairThreads<D>, sizeof(D) == 2 ? 3 : 2) tgv_iter_pair_kernel(const PairArgs<S, D> P)
{
    extern __shared__ __align__(128) unsigned char smem[];
    PairCta<S, D, NB, kPairHaloWarps<D>> C(P, smem);
    const uint32_t it0 = blockIdx.x * P.xrun;
    if (it0 >= (uint32_t)P.it.nitems) return;
    uint64_t* bar = C.bar();
    if (C.t == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init(&bar[2], 1);  // never arrived on: the target of a test-mode wait
        fence_mbar_init();
    }
    uint32_t parity = 0;
    const StridedRuns q{P.xrun, gridDim.x, (uint32_t)P.it.nitems, 0u};
    pair_sweep(C, q, it0, parity, P.wait_test != 0);
}

namespace {

// Items per run, chosen on the host from the level's links (cached per work list
// and grid).  Estimated time of the slowest CTA for run length R:
//   (items it takes) x (1 - f_int x interior + missed halo bytes / item bytes)
// * interior: share of items with hand-overs on both x faces, which skip both
//   x-face halo tasks (the slowest warps of phase A); f_int = 0.12 measured on
//   dense blocks;
// * missed halo bytes: item i is processed at step T(i) = (i / (G R)) R + i % R
//   (G CTAs).  A halo read of the neighbour j hits L2 only when the neighbour's
//   own stream is close in time: |T(j) - T(i)| x G items, with ~80 KB of traffic
//   each, within the ~64 MB of L2 that keeps such data.  A miss costs the
//   neighbour's face layer from DRAM: ~8 KB on a y face (rows of 32 B fetched in
//   longer lines), ~2 KB on a z face, ~16 KB on an x face (a column touches
//   every row of the neighbour's fields); 16-bit storage about 5/8 of that.
// Runs that do not divide the row length of a dense block put y neighbours
// several steps apart and lose to shorter ones.  Candidates 1..16 (divisors of
// typical row lengths), ties to the shorter run.  f_int was measured on the
// 256-thread form; in the FP32 halo-warp form the x-face tasks run on the halo
// warps, and on dense 256^3 its choice (16) stays the fastest (run lengths 1 / 8 /
// 16: 498 / 506 / 471 us).
// 16-bit storage takes no runs: its x-face columns cost half the sectors, the
// split stores of the x = 6 / x = 7 voxels cost more L2 write sectors, and runs
// measured slower (dense 256^3: 607 us per launch without runs, 637 us with 16).
int pair_run_length(const int32_t* nbr, int64_t nb, const int32_t* work, int64_t n, int64_t slots, uint32_t sb)
{
    if (n <= 1 || slots <= 0 || sb != 4) return 1;
    const bool wl = work != nullptr;
    std::vector<int32_t> item_of;
    if (wl) {
        item_of.assign((size_t)nb, -1);
        for (int64_t i = 0; i < n; ++i) item_of[(size_t)work[i]] = (int32_t)i;
    }
    auto brick = [&](int64_t i) -> int32_t { return wl ? work[i] : (int32_t)i; };
    auto item = [&](int32_t b) -> int64_t { return wl ? item_of[(size_t)b] : (int64_t)b; };
    const double item_bytes = (16.0 + 30.0 * sb) * 512.0;
    const double window = 64.0e6 / item_bytes;
    const double scale = sb == 4 ? 1.0 : 0.625;
    const double miss_bytes[3] = {16384.0 * scale, 8192.0 * scale, 2048.0 * scale};  // x, y, z faces
    // sample about 2048 items; the stride is prime to 2 and 3, so samples fall at
    // every position of a run for every candidate length
    int64_t stride = n > 2048 ? n / 2048 : 1;
    while (stride > 1 && (stride % 2 == 0 || stride % 3 == 0)) ++stride;
    static const int kCand[] = {1, 2, 3, 4, 6, 8, 12, 16};
    int best = 1;
    double best_t = 0.0;
    for (int R : kCand) {
        const int64_t nruns = (n + R - 1) / R;
        const int64_t G = nruns < slots ? nruns : slots;
        const double per_cta = (double)((nruns + G - 1) / G) * R;
        auto T = [&](int64_t i) -> int64_t { return (i / (G * R)) * R + i % R; };
        double extra = 0.0;
        int64_t interior = 0, cnt = 0;
        for (int64_t i = 0; i < n; i += stride) {
            ++cnt;
            const int32_t* row = nbr + (size_t)brick(i) * TGV_NNBR;
            const bool from_prev = R > 1 && i % R != 0 && row[NB_MX] == brick(i - 1);
            const bool to_next = R > 1 && (i + 1) % R != 0 && i + 1 < n && row[NB_PX] == brick(i + 1);
            interior += from_prev && to_next;
            const int64_t Ti = T(i);
            for (int k = 0; k < 6; ++k) {
                const int32_t nbk = row[k];
                if (nbk < 0 || nbk >= nb) continue;
                if ((k == NB_MX && from_prev) || (k == NB_PX && to_next)) continue;
                const int64_t j = item(nbk);
                if (j < 0) continue;  // not updated here: its halo reads miss for every R alike
                const int64_t dT = T(j) > Ti ? T(j) - Ti : Ti - T(j);
                if ((double)(dT * G) > window) extra += miss_bytes[k / 2];
            }
        }
        const double t = per_cta * (1.0 - 0.12 * (double)interior / cnt + extra / cnt / item_bytes);
        if (R == 1 || t < best_t) {
            best = R;
            best_t = t;
        }
    }
    return best;
}

template <typename S, typename D, int NB>
tgv_status launch_pair_t(tgv_domain* d, TgvLevel& L, int iters)
{
    const uint32_t SB = sizeof(S), SD = sizeof(D);
    const int npairs = (d->prm.nbins + 1) / 2;
    const PairLayout LY = pair_layout(SB, SD, (uint32_t)npairs);
    const uint32_t tx = LY.tx, stage = LY.stage;
    uint32_t off = LY.end;
    PairArgs<S, D> P;
    P.pn_bytes = LY.pn_bytes;
    P.off_pn = LY.off_pn;
    P.off_hal = LY.off_hal;
    P.off_nbr = LY.off_nbr;
    P.off_bar = LY.off_bar;
    const size_t smem = off;
    auto kern = tgv_iter_pair_kernel<S, D, NB>;
    int per_sm = 0;
    tgv_status st = tgv_kernel_setup((const void*)kern, kPairThreads<D>, smem, &per_sm);
    if (st != TGV_OK) return tgv_fail(d, st, "pair kernel setup (shared memory attribute / occupancy) failed");
    if (per_sm < 1) return tgv_fail(d, TGV_ERR_UNSUPPORTED, "pair iteration kernel does not fit on an SM");
    const int64_t nitems = tgv_work_items(L);
    const int64_t slots = (int64_t)per_sm * d->sm_count;
    if (d->prm.x_run == 0 && (L.xrun == 0 || L.xrun_gen != L.work_gen || L.xrun_slots != slots)) {
        const bool host_ok = (int64_t)L.nbr_host.size() >= L.nb * TGV_NNBR &&
                             (!L.work || (int64_t)L.work_host.size() == nitems);
        L.xrun = host_ok ? pair_run_length(L.nbr_host.data(), L.nb, L.work ? L.work_host.data() : nullptr, nitems,
                                           slots, SB)
                         : 1;
        L.xrun_gen = L.work_gen;
        L.xrun_slots = slots;
    }
    const int R = d->prm.x_run > 0 ? d->prm.x_run : L.xrun;
    const int64_t nruns = (nitems + R - 1) / R;
    const int64_t grid = nruns < slots ? nruns : slots;
    P.xrun = (uint32_t)R;
    P.err = d->err;
    P.wait_budget = tgv_wait_budget(d->prm);
    P.wait_test = d->prm.wait_test;
    P.stage_bytes = stage;
    P.tx_bytes = tx;
    for (int it = 0; it < iters; ++it) {
        P.it = tgv_make_iter_args<S, D>(d, L);
        kern<<<(unsigned)grid, kPairThreads<D>, smem, d->stream>>>(P);
        d->launches++;
        L.cur ^= 1;
    }
    return tgv_cuda_check(d, cudaGetLastError(), "tgv_iter_pair_kernel launch");
}

template <typename S, typename D = S>
tgv_status launch_pair_bins(tgv_domain* d, TgvLevel& L, int iters)
{
    switch (d->prm.nbins) {
    case 8: return launch_pair_t<S, D, 8>(d, L, iters);
    case 10: return launch_pair_t<S, D, 10>(d, L, iters);
    case 12: return launch_pair_t<S, D, 12>(d, L, iters);
    default: return launch_pair_t<S, D, 0>(d, L, iters);
    }
}

}  // namespace

tgv_status tgv_launch_iterations_pair(tgv_domain* d, TgvLevel& L, int iters)
{
    if (tgv_work_items(L) == 0 || iters == 0) return TGV_OK;
    switch (d->prm.storage) {
    case TGV_STORAGE_FP32: return launch_pair_bins<float>(d, L, iters);
    case TGV_STORAGE_BF16: return launch_pair_bins<__nv_bfloat16>(d, L, iters);
    case TGV_STORAGE_FP16: return launch_pair_bins<__half>(d, L, iters);
    case TGV_STORAGE_FX16: return launch_pair_bins<__half, int16_t>(d, L, iters);
    }
    return tgv_fail(d, TGV_ERR_INVALID_ARG, "unknown storage type");
}

extern "C" TGV_API tgv_status tgv_pair_run_length(const int32_t* nbr, int64_t nbricks, const int32_t* work, int64_t nwork,
                                          int64_t slots, int32_t storage, int32_t* run_length)
{
    if (!nbr || nbricks <= 0 || slots <= 0 || !run_length || (work && nwork < 0)) return TGV_ERR_INVALID_ARG;
    if (storage < TGV_STORAGE_FP32 || storage > TGV_STORAGE_FX16) return TGV_ERR_INVALID_ARG;
    const int64_t n = work ? nwork : nbricks;
    if (work) {
        std::vector<uint8_t> seen((size_t)nbricks, 0);
        for (int64_t i = 0; i < nwork; ++i)
            if (work[i] < 0 || work[i] >= nbricks || seen[(size_t)work[i]]++) return TGV_ERR_INVALID_ARG;
    }
    *run_length = pair_run_length(nbr, nbricks, work, n, slots, storage == TGV_STORAGE_FP32 ? 4u : 2u);
    return TGV_OK;
}
