// Serving loop: an open-loop request stream over device-resident source images.
//
// Each request names a source image of a caller-owned device pool, an operation
// (resize / warp / gray) and an output size. The loop runs in real time on the
// host (steady clock):
//   arrival   a request becomes pending at its scheduled arrival time;
//   admission pending requests are admitted in arrival order while the bytes in
//             flight (source + destination) stay within the HBM budget and the
//             output arena (caller-owned device memory) has room for the output;
//   batching  (policy 0) whenever one of the K in-flight slots is free, every
//             admitted request not yet launched -- up to max_batch -- goes into one
//             ragged persistent launch on that slot's stream; new arrivals keep
//             being admitted while earlier batches run, and batches on different
//             streams overlap on the device;
//             (policy 1) every admitted request is launched alone, round-robin over
//             the K streams (the per-image baseline);
//             (policy 2) size-aware: every admitted request of at least direct_px
//             output pixels is launched alone as in policy 1, the smaller ones share
//             ragged launches as in policy 0;
//   completion an event per launch is polled; its requests get their completion
//             time, their bytes leave the budget and their arena space is freed.
// The caller reads outputs from the arena at the offsets reported per request.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <vector>

#include "kr_internal.h"

namespace kr {
namespace {

using Clock = std::chrono::steady_clock;

// First-fit allocator over [0, size) with coalescing free ranges (offset -> length).
class Arena {
  public:
    explicit Arena(uint64_t size) { free_[0] = size; }
    // returns false when no range is large enough
    bool alloc(uint64_t bytes, uint64_t &off)
    {
        bytes = (bytes + 255) & ~uint64_t(255);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                off = it->first;
                const uint64_t rest = it->second - bytes;
                free_.erase(it);
                if (rest) free_[off + bytes] = rest;
                return true;
            }
        }
        return false;
    }
    void release(uint64_t off, uint64_t bytes)
    {
        bytes = (bytes + 255) & ~uint64_t(255);
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }

  private:
    std::map<uint64_t, uint64_t> free_;
};

struct Launch {
    std::vector<int> reqs;
    cudaEvent_t done = nullptr;
    int slot = -1;
};

// Injected host-side failures (kr_debug_set_fault): per site, fail every period-th time.
struct FaultSite {
    std::atomic<int> period{0};
    std::atomic<long long> count{0};
    bool fire()
    {
        const int p = period.load(std::memory_order_relaxed);
        return p > 0 && (count.fetch_add(1, std::memory_order_relaxed) + 1) % p == 0;
    }
};
FaultSite g_fault[4];

}  // namespace
}  // namespace kr

using namespace kr;

extern "C" kr_status kr_serve_run(const kr_request_t *reqs, int32_t n, const kr_serve_config_t *cfg,
                                  kr_serve_result_t *results)
{
    if (n < 0 || (n > 0 && (!reqs || !results)) || !cfg) return KR_ERR_INVALID_ARG;
    if (!cfg->pool || cfg->pool_n < 1 || !cfg->out_arena || cfg->streams < 1 || cfg->streams > 64 ||
        cfg->max_batch < 1 || cfg->policy < 0 || cfg->policy > 2 || cfg->direct_px < 0)
        return KR_ERR_INVALID_ARG;
    if (cfg->policy != 1 && (!cfg->workspaces || cfg->ws_bytes_each < kr_batch_workspace_size(cfg->max_batch)))
        return KR_ERR_NO_SPACE;
    for (int i = 0; i < cfg->pool_n; ++i) {
        const kr_image_t &p = cfg->pool[i];
        if (!p.data || p.channels != 3 || p.dtype != KR_U8 || p.layout != KR_HWC || p.batch != 1)
            return KR_ERR_INVALID_ARG;
    }
    // Validate every request and size its output before anything runs.
    std::vector<uint64_t> out_bytes(n), in_bytes(n);
    for (int i = 0; i < n; ++i) {
        const kr_request_t &r = reqs[i];
        if (r.src_index < 0 || r.src_index >= cfg->pool_n) return KR_ERR_INVALID_ARG;
        if (r.op != KR_OP_RESIZE && r.op != KR_OP_WARP && r.op != KR_OP_GRAY) return KR_ERR_INVALID_ARG;
        const kr_image_t &s = cfg->pool[r.src_index];
        if (r.out_h < 1 || r.out_w < 1 || r.out_h > 65535 || r.out_w > 65535) return KR_ERR_INVALID_ARG;
        if (r.op == KR_OP_GRAY && (r.out_h != s.height || r.out_w != s.width)) return KR_ERR_INVALID_ARG;
        const int dC = r.op == KR_OP_GRAY ? 1 : 3;
        out_bytes[i] = (uint64_t)r.out_h * r.out_w * dC;
        in_bytes[i] = (uint64_t)s.height * s.pitch;
        if (out_bytes[i] > cfg->out_arena_bytes) return KR_ERR_NO_SPACE;
        if (cfg->hbm_budget_bytes && in_bytes[i] + out_bytes[i] > cfg->hbm_budget_bytes) return KR_ERR_NO_SPACE;
        if (!std::isfinite(r.t_arrival) || (i > 0 && r.t_arrival < reqs[i - 1].t_arrival)) return KR_ERR_INVALID_ARG;
        if (r.op == KR_OP_WARP)
            for (int k = 0; k < 6; ++k)
                if (!std::isfinite(r.M[k])) return KR_ERR_INVALID_ARG;
    }

    const int K = cfg->streams;
    std::vector<cudaStream_t> streams(K, nullptr);
    std::vector<cudaEvent_t> event_pool;
    kr_status status = KR_OK;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < K && e == cudaSuccess; ++k) e = cudaStreamCreateWithFlags(&streams[k], cudaStreamNonBlocking);
    const int n_events = cfg->policy == 0 ? K : std::min(4096, std::max(K, n)) + (cfg->policy == 2 ? K : 0);
    for (int k = 0; k < n_events && e == cudaSuccess; ++k) {
        cudaEvent_t ev;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) event_pool.push_back(ev);
    }

    Arena arena(cfg->out_arena_bytes);
    FaultSite &f_submit = g_fault[KR_FAULT_SUBMIT], &f_event = g_fault[KR_FAULT_EVENT], &f_admit = g_fault[KR_FAULT_ADMIT];
    std::vector<uint64_t> out_off(n, 0);
    std::deque<int> pending, admitted, small;   // small: policy 2's requests waiting for a batch slot
    std::deque<Launch> inflight;
    std::vector<int> slot_busy(K, 0);
    std::vector<kr_work_t> work;
    work.reserve(cfg->max_batch);
    uint64_t bytes_in_flight = 0;
    int next_arrival = 0, done = 0, rr = 0;
    const Clock::time_point t0 = Clock::now();
    auto now_s = [&] { return std::chrono::duration<double>(Clock::now() - t0).count(); };
    for (int i = 0; i < n; ++i) {
        results[i].t_admit = results[i].t_launch = results[i].t_done = -1.0;
        results[i].out_offset = -1;
        results[i].status = KR_OK;
    }

    // one request through its single-image call
    auto launch_alone = [&](const kr_work_t &w, cudaStream_t s) -> kr_status {
        if (f_submit.fire()) return KR_ERR_CUDA;
        if (w.op == KR_OP_RESIZE) return kr_resize_bilinear(&w.src, &w.dst, nullptr, (kr_stream_t)s);
        if (w.op == KR_OP_WARP) return kr_warp_affine(&w.src, &w.dst, w.M, nullptr, (kr_stream_t)s);
        return kr_rgb_to_gray(&w.src, &w.dst, (kr_stream_t)s);
    };
    auto make_work = [&](int i, kr_work_t &w) {
        const kr_request_t &r = reqs[i];
        std::memset(&w, 0, sizeof(w));
        w.op = r.op;
        w.src = cfg->pool[r.src_index];
        kr_image_t &d = w.dst;
        d.data = (uint8_t *)cfg->out_arena + out_off[i];
        d.height = r.out_h;
        d.width = r.out_w;
        d.channels = r.op == KR_OP_GRAY ? 1 : 3;
        d.dtype = KR_U8;
        d.layout = KR_HWC;
        d.batch = 1;
        d.pitch = (int64_t)r.out_w * d.channels;
        std::memcpy(w.M, r.M, sizeof(w.M));
    };

    // a request leaves the run: completed (td >= 0) or dropped with status st
    auto finish = [&](int i, double td, kr_status st) {
        results[i].t_done = td;
        results[i].status = st;
        bytes_in_flight -= in_bytes[i] + out_bytes[i];
        if (st != KR_OK || !cfg->retain_outputs) arena.release(out_off[i], out_bytes[i]);
        if (st != KR_OK) {
            results[i].t_launch = -1.0;
            results[i].out_offset = -1;
        }
        ++done;
    };
    // a launch whose completion cannot be tracked by an event: wait for its stream
    auto complete_now = [&](const std::vector<int> &ids, cudaStream_t s) -> cudaError_t {
        const cudaError_t q = cudaStreamSynchronize(s);
        if (q == cudaSuccess) {
            const double td = now_s();
            for (int i : ids) finish(i, td, KR_OK);
        }
        return q;
    };

    while (status == KR_OK && done < n) {
        const double t = now_s();
        // arrivals
        while (next_arrival < n && reqs[next_arrival].t_arrival <= t) pending.push_back(next_arrival++);
        // completions
        for (auto it = inflight.begin(); it != inflight.end();) {
            const cudaError_t q = cudaEventQuery(it->done);
            if (q == cudaErrorNotReady) { ++it; continue; }
            if (q != cudaSuccess) { e = q; status = KR_ERR_CUDA; break; }
            const double td = now_s();
            for (int i : it->reqs) finish(i, td, KR_OK);
            if (it->slot >= 0) slot_busy[it->slot] = 0;
            event_pool.push_back(it->done);
            it = inflight.erase(it);
        }
        if (status != KR_OK) break;
        // admission, in arrival order
        bool arena_full = false;
        while (!pending.empty()) {
            const int i = pending.front();
            const uint64_t need = in_bytes[i] + out_bytes[i];
            if (cfg->hbm_budget_bytes && bytes_in_flight + need > cfg->hbm_budget_bytes) break;
            uint64_t off;
            if (f_admit.fire()) break;   // an injected failure: the request waits, as for a full arena
            if (!arena.alloc(out_bytes[i], off)) {
                arena_full = true;
                break;
            }
            out_off[i] = off;
            bytes_in_flight += need;
            results[i].t_admit = now_s();
            results[i].out_offset = (int64_t)off;
            pending.pop_front();
            admitted.push_back(i);
        }
        // nothing runs and the head request can never be admitted: the arena is full of
        // retained outputs
        if (arena_full && !pending.empty() && admitted.empty() && small.empty() && inflight.empty() && next_arrival == n) {
            status = KR_ERR_NO_SPACE;
            break;
        }
        // launches
        const int64_t direct_px = cfg->direct_px > 0 ? cfg->direct_px : (int64_t)1 << 20;
        if (cfg->policy != 0) {
            // per-image launches, round-robin over the streams, each tracked by its own event:
            // every admitted request (policy 1), or those of at least direct_px output pixels
            // (policy 2, the others wait for a batch slot)
            while (!admitted.empty() && !event_pool.empty() && status == KR_OK) {
                const int i = admitted.front();
                admitted.pop_front();
                kr_work_t w;
                make_work(i, w);
                if (cfg->policy == 2 && (int64_t)w.dst.width * w.dst.height < direct_px) {
                    small.push_back(i);
                    continue;
                }
                cudaStream_t st_s = streams[rr];
                rr = (rr + 1) % K;
                const double tl = now_s();
                const kr_status st = launch_alone(w, st_s);
                results[i].t_launch = tl;
                if (st != KR_OK) {
                    finish(i, -1.0, st);
                    continue;
                }
                Launch L;
                L.reqs.push_back(i);
                L.done = event_pool.back();
                event_pool.pop_back();
                e = f_event.fire() ? cudaErrorUnknown : cudaEventRecord(L.done, st_s);
                if (e != cudaSuccess) {
                    event_pool.push_back(L.done);
                    e = complete_now(L.reqs, st_s);
                    if (e != cudaSuccess) status = KR_ERR_CUDA;
                    continue;
                }
                inflight.push_back(std::move(L));
            }
            if (status != KR_OK) break;
        }
        if (cfg->policy != 1) {
            // ragged batches: whenever a slot is free, the waiting requests (all admitted ones for
            // policy 0, the small ones for policy 2) -- up to max_batch -- share one launch on
            // the slot's stream
            std::deque<int> &q = cfg->policy == 0 ? admitted : small;
            for (int k = 0; k < K && !q.empty() && !event_pool.empty(); ++k) {
                if (slot_busy[k]) continue;
                Launch L;
                L.slot = k;
                work.clear();
                const double tl = now_s();
                while (!q.empty() && (int)L.reqs.size() < cfg->max_batch) {
                    const int i = q.front();
                    q.pop_front();
                    kr_work_t w;
                    make_work(i, w);
                    L.reqs.push_back(i);
                    work.push_back(w);
                }
                void *ws = (uint8_t *)cfg->workspaces + (size_t)k * cfg->ws_bytes_each;
                const kr_status st = f_submit.fire() ? KR_ERR_CUDA
                                                     : kr_batch_submit(work.data(), (int32_t)work.size(), ws,
                                                                       cfg->ws_bytes_each, nullptr,
                                                                       (kr_stream_t)streams[k]);
                for (int i : L.reqs) results[i].t_launch = tl;
                if (st != KR_OK) {
                    // the launch failed: its requests are dropped
                    for (int i : L.reqs) finish(i, -1.0, st);
                    continue;
                }
                L.done = event_pool.back();
                event_pool.pop_back();
                e = f_event.fire() ? cudaErrorUnknown : cudaEventRecord(L.done, streams[k]);
                if (e != cudaSuccess) {
                    event_pool.push_back(L.done);
                    e = complete_now(L.reqs, streams[k]);
                    if (e != cudaSuccess) { status = KR_ERR_CUDA; break; }
                    continue;
                }
                slot_busy[k] = 1;
                inflight.push_back(std::move(L));
            }
        }
    }
    if (status == KR_ERR_CUDA) set_last_error("kr_serve_run", e);
    for (auto &s : streams)
        if (s) cudaStreamSynchronize(s);
    // a run that stopped early drops every request that did not complete
    if (status != KR_OK)
        for (int i = 0; i < n; ++i)
            if (results[i].t_done < 0) {
                results[i].status = status;
                results[i].t_launch = -1.0;
                results[i].out_offset = -1;
            }
    for (auto &L : inflight) event_pool.push_back(L.done);
    for (auto ev : event_pool) cudaEventDestroy(ev);
    for (auto &s : streams)
        if (s) cudaStreamDestroy(s);
    return status;
}

extern "C" kr_status kr_debug_set_fault(int32_t site, int32_t period)
{
    if (site < KR_FAULT_SUBMIT || site > KR_FAULT_ADMIT || period < 0) return KR_ERR_INVALID_ARG;
    kr::g_fault[site].period.store(period, std::memory_order_relaxed);
    kr::g_fault[site].count.store(0, std::memory_order_relaxed);
    return KR_OK;
}
