// vkt_tune.cu -- the autotuner's memory: the launch choices (evaluation path, z chunk of a
// brick, batch brick extent and grid) that the first call of each call shape measured, kept
// in memory and, when the environment names a file in VKT_AUTOTUNE_CACHE, in that JSON file
// (read at the first lookup, rewritten after every new choice).
//
// File format (JSON, one entry per line so that it is also read back line by line):
//   {"vkt_autotune": 1, "entries": [
//   {"key": "<call shape>", "path": P, "zchunk": Z, "ms": T},
//   ...
//   ]}
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "vkt_internal.h"

namespace vkt {
namespace {

std::mutex g_tune_mutex;
std::map<std::string, TuneChoice> g_choices;
bool g_env_loaded = false;
int g_enabled = -1;   // -1: not yet read from VKT_AUTOTUNE

const char* env_cache() { return std::getenv("VKT_AUTOTUNE_CACHE"); }

// Parses one entry line; false if it holds no entry.
bool parse_entry(const char* line, std::string* key, TuneChoice* c)
{
    const char* k = std::strstr(line, "\"key\": \"");
    if (!k) return false;
    k += 8;
    const char* e = std::strchr(k, '"');
    if (!e) return false;
    const char* p = std::strstr(e, "\"path\": ");
    const char* z = std::strstr(e, "\"zchunk\": ");
    const char* m = std::strstr(e, "\"ms\": ");
    if (!p || !z || !m) return false;
    key->assign(k, e);
    c->path = static_cast<int>(std::strtol(p + 8, nullptr, 10));
    c->zchunk = static_cast<int>(std::strtol(z + 10, nullptr, 10));
    c->ms = std::strtof(m + 6, nullptr);
    return true;
}

// Reads the entries of a cache file into the table (caller holds the mutex).
bool load_locked(const char* path, int* added)
{
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    char line[1024];
    int n = 0;
    while (std::fgets(line, sizeof(line), f)) {
        std::string key;
        TuneChoice c;
        if (parse_entry(line, &key, &c)) {
            g_choices[key] = c;
            ++n;
        }
    }
    std::fclose(f);
    if (added) *added = n;
    return true;
}

bool save_locked(const char* path)
{
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "w");
    if (!f) return false;
    std::fprintf(f, "{\"vkt_autotune\": 1, \"entries\": [\n");
    size_t i = 0;
    for (const auto& kv : g_choices) {
        std::fprintf(f, "{\"key\": \"%s\", \"path\": %d, \"zchunk\": %d, \"ms\": %.6g}%s\n",
                     kv.first.c_str(), kv.second.path, kv.second.zchunk, kv.second.ms,
                     ++i < g_choices.size() ? "," : "");
    }
    std::fprintf(f, "]}\n");
    const bool ok = std::fclose(f) == 0;
    return ok && std::rename(tmp.c_str(), path) == 0;
}

void load_env_locked()
{
    if (g_env_loaded) return;
    g_env_loaded = true;
    if (const char* p = env_cache()) load_locked(p, nullptr);
}

}  // namespace

bool autotune_enabled()
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    if (g_enabled < 0) {
        const char* e = std::getenv("VKT_AUTOTUNE");
        g_enabled = (e && std::strcmp(e, "0") == 0) ? 0 : 1;
    }
    return g_enabled != 0;
}

bool autotune_lookup(const char* key, TuneChoice* c)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    load_env_locked();
    auto it = g_choices.find(key);
    if (it == g_choices.end()) return false;
    *c = it->second;
    return true;
}

void autotune_store(const char* key, const TuneChoice& c)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    load_env_locked();
    g_choices[key] = c;
    if (const char* p = env_cache()) save_locked(p);
}

bool stream_capturing(cudaStream_t stream)
{
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &st) != cudaSuccess) {
        cudaGetLastError();
        return true;   // cannot tell: do not time
    }
    return st != cudaStreamCaptureStatusNone;
}

}  // namespace vkt

using namespace vkt;

extern "C" {

vktError vktAutotuneSetEnabled(int32_t enabled)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_enabled = enabled ? 1 : 0;
    return VKT_NO_ERROR;
}

vktError vktAutotuneGetEnabled(int32_t* enabled)
{
    if (!enabled) return VKT_ERROR_INVALID_VALUE;
    *enabled = autotune_enabled() ? 1 : 0;
    return VKT_NO_ERROR;
}

vktError vktAutotuneClear(void)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_choices.clear();
    g_env_loaded = true;   // a cleared table does not reload the environment's file
    return VKT_NO_ERROR;
}

vktError vktAutotuneGetCount(int32_t* count)
{
    if (!count) return VKT_ERROR_INVALID_VALUE;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    load_env_locked();
    *count = static_cast<int32_t>(g_choices.size());
    return VKT_NO_ERROR;
}

vktError vktAutotuneSave(const char* path)
{
    if (!path) return VKT_ERROR_INVALID_VALUE;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    return save_locked(path) ? VKT_NO_ERROR : VKT_ERROR_INVALID_VALUE;
}

vktError vktAutotuneLoad(const char* path)
{
    if (!path) return VKT_ERROR_INVALID_VALUE;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    return load_locked(path, nullptr) ? VKT_NO_ERROR : VKT_ERROR_INVALID_VALUE;
}

}  // extern "C"
