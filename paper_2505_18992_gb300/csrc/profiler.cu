// Launch counter and optional per-kernel CUDA-event timing (see profiler.h).
#include <stdint.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/vpgs.h"
#include "profiler.h"

namespace vpgs {
namespace {

struct Record {
    const char *name;
    cudaEvent_t start, stop;
};

std::mutex g_mu;
int64_t g_launches = 0;
bool g_enabled = false;
std::vector<Record> g_records;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

}  // namespace

void prof_begin(const char *name, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_mu);
    ++g_launches;
    if (!g_enabled) return;
    Record r{name, take_event(), take_event()};
    cudaEventRecord(r.start, s);
    g_records.push_back(r);
}

void prof_end(cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_enabled || g_records.empty()) return;
    cudaEventRecord(g_records.back().stop, s);
}

}  // namespace vpgs

extern "C" {

int64_t vpgs_launch_count(void) {
    std::lock_guard<std::mutex> lk(vpgs::g_mu);
    return vpgs::g_launches;
}

void vpgs_profile_enable(int32_t on) {
    std::lock_guard<std::mutex> lk(vpgs::g_mu);
    vpgs::g_enabled = on != 0;
}

int32_t vpgs_profile_collect(char *names, size_t name_bytes, int64_t *launches, double *total_ms,
                             int32_t max_entries) {
    std::lock_guard<std::mutex> lk(vpgs::g_mu);
    std::map<std::string, std::pair<int64_t, double>> agg;
    std::vector<std::string> order;
    for (auto &r : vpgs::g_records) {
        float ms = 0.f;
        cudaEventSynchronize(r.stop);
        cudaEventElapsedTime(&ms, r.start, r.stop);
        auto it = agg.find(r.name);
        if (it == agg.end()) {
            order.push_back(r.name);
            agg[r.name] = {1, (double)ms};
        } else {
            it->second.first += 1;
            it->second.second += ms;
        }
        vpgs::g_pool.push_back(r.start);
        vpgs::g_pool.push_back(r.stop);
    }
    vpgs::g_records.clear();
    int32_t n = 0;
    size_t pos = 0;
    for (auto &nm : order) {
        if (n >= max_entries) break;
        if (names) {
            if (pos + nm.size() + 1 > name_bytes) break;
            memcpy(names + pos, nm.c_str(), nm.size() + 1);
            pos += nm.size() + 1;
        }
        if (launches) launches[n] = agg[nm].first;
        if (total_ms) total_ms[n] = agg[nm].second;
        ++n;
    }
    return n;
}

}  // extern "C"
