// autotune.cu -- picks the fastest execution schedule for a network.
//
// Candidates: per-step launches with warp-per-chunk delivery at 128 and 256
// threads per block, per-step launches with thread-per-synapse delivery at
// 128 and 256, the persistent kernel, the persistent target-tiled kernel
// when the network has the grouped layout and its tile fits, and the
// persistent owner-windowed kernel when a window fits.  Each candidate
// runs `trial_steps` steps from the same snapshot of the dynamic state, timed
// with CUDA events on the caller's stream; the state is restored afterwards,
// so tuning never changes the simulation.  The choice is cached in a text
// file, one line per key: the network's shape, weight type, layout, rate and
// the GPU.
#include "snn.h"
#include "snn_internal.h"

#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

namespace {

snn_status afail(snn_status s, const std::string& m) {
    snn::set_last_error(m.c_str());
    return s;
}

std::string tune_key(snn_net* net) {
    uint32_t N = 0, K = 0, D = 0;
    uint64_t bytes = 0;
    snn_get_dims(net, &N, &K, &D, &bytes);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp p;
    cudaGetDeviceProperties(&p, dev);
    char buf[512];
    const snn_config* c = snn_config_of(net);
    snprintf(buf, sizeof buf, "N=%u;K=%u;D=%u;kernel=%d;w=%d;layout=%d;rate=%.2f;ext=%.1f;gpu=%s;sm=%d", N, K, D,
             c->kernel, c->weight_dtype, c->table_layout, c->imposed_rate_hz, c->ext_rate_hz, p.name,
             p.multiProcessorCount);
    for (char* q = buf; *q; ++q)
        if (*q == ' ') *q = '_';
    return buf;
}

bool cache_lookup(const char* path, const std::string& key, int* schedule, int* block) {
    if (!path) return false;
    FILE* f = fopen(path, "r");
    if (!f) return false;
    char line[768];
    bool hit = false;
    while (fgets(line, sizeof line, f)) {
        char k[600];
        int s = 0, b = 0;
        if (sscanf(line, "%599s %d %d", k, &s, &b) == 3 && key == k) {
            *schedule = s;
            *block = b;
            hit = true;  // the last entry for the key wins
        }
    }
    fclose(f);
    return hit;
}

void cache_store(const char* path, const std::string& key, int schedule, int block) {
    if (!path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d %d\n", key.c_str(), schedule, block);
    fclose(f);
}

}  // namespace

extern "C" {

snn_status snn_autotune(snn_net* net, uint32_t trial_steps, const char* cache_path, int32_t* schedule, int32_t* block,
                        double* best_ms_per_step, void* stream) {
    if (!net || trial_steps == 0) return afail(SNN_EINVAL, "net is NULL or trial_steps is 0");
    snn::NvtxRange range("snn_autotune");
    const std::string key = tune_key(net);
    int s = 0, b = 0;
    if (cache_lookup(cache_path, key, &s, &b) && snn_set_schedule(net, s, b) == SNN_OK) {
        if (schedule) *schedule = s;
        if (block) *block = b;
        if (best_ms_per_step) *best_ms_per_step = -1.0;  // from the cache, not measured
        return SNN_OK;
    }
    cudaStream_t st = (cudaStream_t)stream;
    snn_stats before{};
    snn_status e0 = snn_get_stats(net, &before, stream);
    if (e0 != SNN_OK) return e0;
    size_t n = 0;
    snn_status e = snn_snapshot(net, nullptr, 0, &n, stream);
    if (e != SNN_OK) return e;
    std::vector<char> snap(n);
    e = snn_snapshot(net, snap.data(), n, &n, stream);
    if (e != SNN_OK) return e;
    const int cand[][2] = {{0, 128}, {0, 256}, {1, 128}, {1, 256}, {2, 0}, {3, 0}, {4, 0}, {5, 0}};
    cudaEvent_t a, z;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&z) != cudaSuccess)
        return afail(SNN_ECUDA, "cudaEventCreate failed");
    double best = 1e300;
    int bs = -1, bb = 0;
    for (auto& c : cand) {
        if (snn_set_schedule(net, c[0], c[1]) != SNN_OK) continue;  // e.g. no grouped layout
        if ((e = snn_restore(net, snap.data(), n, stream)) != SNN_OK) break;
        // trials record no spikes: the raster counter sits at the capacity
        if (snn_set_raster_count(net, before.raster_capacity, st) != cudaSuccess) {
            e = afail(SNN_ECUDA, "parking the raster counter failed");
            break;
        }
        if ((e = snn_step(net, 2, stream)) != SNN_OK) break;  // warm-up
        cudaEventRecord(a, st);
        if ((e = snn_step(net, trial_steps, stream)) != SNN_OK) break;
        cudaEventRecord(z, st);
        if (cudaEventSynchronize(z) != cudaSuccess) {
            e = afail(SNN_ECUDA, "autotune trial failed");
            break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, a, z);
        if (ms < best) {
            best = ms;
            bs = c[0];
            bb = c[1];
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(z);
    snn_status r = snn_restore(net, snap.data(), n, stream);
    if (e != SNN_OK) return e;
    if (r != SNN_OK) return r;
    if (snn_set_raster_count(net, before.raster_count, st) != cudaSuccess)  // the raster is kept as it was
        return afail(SNN_ECUDA, "restoring the raster count failed");
    if (bs < 0) return afail(SNN_EINVAL, "no schedule could run");
    snn_set_schedule(net, bs, bb);
    cache_store(cache_path, key, bs, bb);
    if (schedule) *schedule = bs;
    if (block) *block = bb;
    if (best_ms_per_step) *best_ms_per_step = best / trial_steps;
    return SNN_OK;
}

}  // extern "C"
