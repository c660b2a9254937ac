// Kernel profiler (see profile.cuh) and its C ABI.
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>

#include "kernels.cuh"
#include "profile.cuh"

namespace msb {

namespace {
struct Stat {
    int64_t launches = 0;
    double ms = 0, bytes = 0, flops = 0;
};
struct Pending {
    int id;
    cudaEvent_t e0, e1;
    double bytes, flops;
};
std::atomic<bool> g_on{false};
std::mutex g_mu;
std::vector<std::string> g_names;
std::map<std::string, int> g_ids;
std::vector<Stat> g_stats;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t get_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}
}  // namespace

bool prof_on() { return g_on.load(std::memory_order_relaxed); }

ProfScope::ProfScope(const char* name, cudaStream_t s, double alg_bytes, double alg_flops)
    : st(s), bytes(alg_bytes), flops(alg_flops) {
    if (!prof_on()) return;
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_ids.find(name);
    if (it == g_ids.end()) {
        id = int(g_names.size());
        g_ids[name] = id;
        g_names.push_back(name);
        g_stats.emplace_back();
    } else {
        id = it->second;
    }
    e0 = get_event();
    e1 = get_event();
    if (!e0 || !e1) { id = -1; return; }
    cudaEventRecord(e0, st);
}

void ProfScope::done() {
    if (id < 0) return;
    cudaEventRecord(e1, st);
    std::lock_guard<std::mutex> lk(g_mu);
    g_pending.push_back(Pending{id, e0, e1, bytes, flops});
    id = -1;
}

void prof_patch_last(const char* name, double alg_bytes, double alg_flops) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_ids.find(name);
    if (it == g_ids.end()) return;
    for (size_t i = g_pending.size(); i-- > 0;) {
        if (g_pending[i].id == it->second) {
            g_pending[i].bytes = alg_bytes;
            g_pending[i].flops = alg_flops;
            return;
        }
    }
}

void prof_collect() {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& p : g_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.e1) == cudaSuccess && cudaEventElapsedTime(&ms, p.e0, p.e1) == cudaSuccess) {
            Stat& s = g_stats[p.id];
            s.launches += 1;
            s.ms += ms;
            s.bytes += p.bytes;
            s.flops += p.flops;
        }
        g_pool.push_back(p.e0);
        g_pool.push_back(p.e1);
    }
    g_pending.clear();
    cudaGetLastError();
}

}  // namespace msb

extern "C" void msb_profile_enable(int on) {
    msb::prof_collect();
    msb::g_on.store(on != 0);
}

extern "C" void msb_profile_reset(void) {
    msb::prof_collect();
    std::lock_guard<std::mutex> lk(msb::g_mu);
    for (auto& s : msb::g_stats) s = msb::Stat{};
}

extern "C" int msb_profile_read(msb_kernel_stat* out, int max) {
    msb::prof_collect();
    std::lock_guard<std::mutex> lk(msb::g_mu);
    int n = 0;
    for (size_t i = 0; i < msb::g_names.size() && (out == nullptr || n < max); ++i) {
        if (msb::g_stats[i].launches == 0) continue;
        if (out) {
            std::memset(&out[n], 0, sizeof(msb_kernel_stat));
            std::strncpy(out[n].name, msb::g_names[i].c_str(), sizeof(out[n].name) - 1);
            out[n].launches = msb::g_stats[i].launches;
            out[n].ms = msb::g_stats[i].ms;
            out[n].alg_bytes = msb::g_stats[i].bytes;
            out[n].alg_flops = msb::g_stats[i].flops;
        }
        ++n;
    }
    return n;
}
