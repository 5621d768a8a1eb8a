// Process-wide instrumentation: kernel-launch counter and event timing of grouped GEMMs.
#include <algorithm>
#include <mutex>
#include <vector>

#include "plans.h"

namespace pd {

thread_local int g_sm_cap = 0;

namespace {
struct PinnedWords {
    int* p = nullptr;
    int n = 0;
    ~PinnedWords() {
        if (p) cudaFreeHost(p);
    }
};
thread_local PinnedWords g_flags;
}  // namespace

int* sweep_flags_host(int n) {
    if (g_flags.n < n) {
        if (g_flags.p) PD_CK(cudaFreeHost(g_flags.p));
        g_flags.p = nullptr;
        g_flags.n = 0;
        PD_CK(cudaMallocHost(&g_flags.p, sizeof(int) * (size_t)n));
        g_flags.n = n;
    }
    return g_flags.p;
}

std::atomic<long long> g_launches{0};
std::atomic<long long> g_fallbacks{0};
std::atomic<long long> g_emu_fallbacks{0};
thread_local int g_prof_class = PROF_MV;

namespace {
struct Rec {
    cudaEvent_t a, b;
    int cls;
    double flops;
};
std::mutex g_mu;
std::atomic<bool> g_on{false};
std::vector<Rec> g_pending;
long long g_svd_calls = 0, g_svd_sweeps = 0, g_svd_block = 0, g_svd_f64 = 0, g_svd_rows = 0, g_svd_bonds = 0;
double g_svd_ms = 0.0, g_svd_block_ms = 0.0, g_svd_f64_ms = 0.0, g_svd_block_flops = 0.0;
double g_svd_block_alg_flops = 0.0, g_svd_block_alg_bytes = 0.0;
long long g_rot_hist[48] = {0};
double g_ms[4] = {0, 0, 0, 0}, g_fl[4] = {0, 0, 0, 0};
long long g_n[4] = {0, 0, 0, 0};
}  // namespace

bool prof_on() { return g_on.load(std::memory_order_relaxed); }

void prof_fallback() { g_fallbacks.fetch_add(1); }
void prof_emu_fallback() { g_emu_fallbacks.fetch_add(1); }

void* prof_start(cudaStream_t st) {
    cudaEvent_t* ev = new cudaEvent_t[2];
    PD_CK(cudaEventCreate(&ev[0]));
    PD_CK(cudaEventCreate(&ev[1]));
    PD_CK(cudaEventRecord(ev[0], st));
    return ev;
}

void prof_stop(void* token, cudaStream_t st, int cls, double flops) {
    cudaEvent_t* ev = static_cast<cudaEvent_t*>(token);
    PD_CK(cudaEventRecord(ev[1], st));
    std::lock_guard<std::mutex> lk(g_mu);
    g_pending.push_back({ev[0], ev[1], cls, flops});
    delete[] ev;
}

void prof_svd(int sweeps, double ms, int kind, int max_rows, double flops, const int* rot_hist, int nhist,
              int bonds, double alg_flops, double alg_bytes) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_svd_calls += 1;
    g_svd_bonds += bonds;
    g_svd_sweeps += sweeps;
    g_svd_ms += ms;
    if (kind == 1) {
        g_svd_block += 1;
        g_svd_block_ms += ms;
        g_svd_block_flops += flops;
        g_svd_block_alg_flops += alg_flops;
        g_svd_block_alg_bytes += alg_bytes;
    }
    if (kind == 2) g_svd_f64 += 1, g_svd_f64_ms += ms;
    g_svd_rows = std::max<long long>(g_svd_rows, max_rows);
    for (int i = 0; rot_hist && i < nhist && i < 48; ++i) g_rot_hist[i] += rot_hist[i];
}

}  // namespace pd

using namespace pd;

extern "C" {

void dmrg_profile_enable(int on) { g_on.store(on != 0); }

void dmrg_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    cudaDeviceSynchronize();
    for (auto& r : g_pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    g_pending.clear();
    for (int i = 0; i < 4; ++i) g_ms[i] = g_fl[i] = 0.0, g_n[i] = 0;
    g_svd_calls = g_svd_sweeps = g_svd_block = g_svd_f64 = g_svd_rows = g_svd_bonds = 0;
    g_svd_ms = g_svd_block_ms = g_svd_f64_ms = g_svd_block_flops = 0.0;
    g_svd_block_alg_flops = g_svd_block_alg_bytes = 0.0;
    for (auto& x : g_rot_hist) x = 0;
    g_launches.store(0);
    g_fallbacks.store(0);
    g_emu_fallbacks.store(0);
}

dmrg_status dmrg_profile_read(dmrg_profile* out) {
    if (!out) return DMRG_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    if (cudaDeviceSynchronize() != cudaSuccess) return DMRG_ERR_CUDA;
    for (auto& r : g_pending) {
        float ms = 0.f;
        if (r.cls >= 0 && r.cls < 4 && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            g_ms[r.cls] += ms;
            g_fl[r.cls] += r.flops;
            g_n[r.cls] += 1;
        }
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    g_pending.clear();
    out->launches = g_launches.load();
    out->mv_gemm_launches = g_n[PROF_MV];
    out->mv_gemm_ms = g_ms[PROF_MV];
    out->mv_gemm_flops = g_fl[PROF_MV];
    out->env_gemm_launches = g_n[PROF_ENV];
    out->env_gemm_ms = g_ms[PROF_ENV];
    out->env_gemm_flops = g_fl[PROF_ENV];
    out->f64_gemm_launches = g_n[PROF_F64];
    out->f64_gemm_ms = g_ms[PROF_F64];
    out->f64_gemm_flops = g_fl[PROF_F64];
    out->f32_gemm_launches = g_n[PROF_F32];
    out->f32_gemm_ms = g_ms[PROF_F32];
    out->f32_gemm_flops = g_fl[PROF_F32];
    out->svd_calls = g_svd_calls;
    out->svd_bonds = g_svd_bonds;
    out->svd_sweeps = g_svd_sweeps;
    out->svd_ms = g_svd_ms;
    out->svd_block_calls = g_svd_block;
    out->svd_fp64_calls = g_svd_f64;
    out->svd_block_ms = g_svd_block_ms;
    out->svd_fp64_ms = g_svd_f64_ms;
    out->svd_max_rows = g_svd_rows;
    out->svd_fp64_fallbacks = g_fallbacks.load();
    out->svd_block_flops = g_svd_block_flops;
    out->svd_block_alg_flops = g_svd_block_alg_flops;
    out->svd_block_alg_bytes = g_svd_block_alg_bytes;
    for (int i = 0; i < 48; ++i) out->svd_rot_hist[i] = g_rot_hist[i];
    out->emu_fallbacks = g_emu_fallbacks.load();
    tune_stats(&out->tune_classes, &out->tune_changed);
    return DMRG_OK;
}

}  // extern "C"
