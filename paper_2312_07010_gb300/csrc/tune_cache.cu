// tune_cache.cu -- the autotuners' cache: one line per problem class,
//   <key> <four integers> <microseconds per step>
// where <key> names the device (name and SM count) and the class: for a single problem
// dims, n, bc, dtype and scheme, with <kernel> <depth> <variant> <chunk>; for a batch
// its workload class (acs_batch_autotune), with <ctas per SM> <blocks per ticket>
// <block order> and 0 for single steps, else depth | unit order << 3 | rows per unit << 4
// of the temporally blocked kernel.
// The file is $ACS_TUNE_CACHE, else $HOME/.cache/acs_tune.txt; missing or
// unreadable files simply mean "not cached".  Later lines win.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>

#include <sys/stat.h>

#include "acs_host.h"

namespace acs {
namespace {

std::mutex g_mu;

std::string cache_path() {
    if (const char* p = std::getenv("ACS_TUNE_CACHE")) return p;
    if (const char* h = std::getenv("HOME")) return std::string(h) + "/.cache/acs_tune.txt";
    return std::string();
}

std::string device_prefix() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceProp prop;
    std::string name = "gpu";
    if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
    for (char& ch : name)
        if (ch == ' ') ch = '_';
    return name + "/sm" + std::to_string(sms);
}

// Last line of the cache whose key is `key`: its four integers.
bool lookup_line(const std::string& key, int* v4) {
    const std::string path = cache_path();
    if (path.empty()) return false;
    std::lock_guard<std::mutex> lock(g_mu);
    FILE* f = std::fopen(path.c_str(), "r");
    if (!f) return false;
    char line[512], k[300];
    bool found = false;
    while (std::fgets(line, sizeof(line), f)) {
        int a, b, c, d;
        double us;
        if (std::sscanf(line, "%299s %d %d %d %d %lf", k, &a, &b, &c, &d, &us) == 6 && key == k) {
            v4[0] = a; v4[1] = b; v4[2] = c; v4[3] = d;
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

void store_line(const std::string& key, const int* v4, double us) {
    const std::string path = cache_path();
    if (path.empty()) return;
    std::lock_guard<std::mutex> lock(g_mu);
    FILE* f = std::fopen(path.c_str(), "a");
    if (!f) {
        // create the missing directories of the path, one component at a time
        const std::string dir = path.substr(0, path.find_last_of('/'));
        for (size_t i = 1; i <= dir.size(); ++i)
            if (i == dir.size() || dir[i] == '/') (void)mkdir(dir.substr(0, i).c_str(), 0755);
        f = std::fopen(path.c_str(), "a");
        if (!f) return;
    }
    std::fprintf(f, "%s %d %d %d %d %.3f\n", key.c_str(), v4[0], v4[1], v4[2], v4[3], us);
    std::fclose(f);
}

std::string make_key(int dims, const int64_t* n, int bc, int dtype, int scheme) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceProp prop;
    std::string name = "gpu";
    if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
    for (char& ch : name)
        if (ch == ' ') ch = '_';
    char buf[256];
    std::snprintf(buf, sizeof(buf), "%s/sm%d/d%d/n%lldx%lldx%lld/bc%d/t%d/s%d", name.c_str(), sms, dims,
                  (long long)n[0], (long long)(dims > 1 ? n[1] : 1), (long long)(dims > 2 ? n[2] : 1), bc, dtype,
                  scheme);
    return buf;
}

}  // namespace

bool tune_cache_lookup(int dims, const int64_t* n, int bc, int dtype, int scheme, int* kernel, int* depth,
                       int* variant, int* chunk) {
    int v[4];
    if (!lookup_line(make_key(dims, n, bc, dtype, scheme), v)) return false;
    *kernel = v[0]; *depth = v[1]; *variant = v[2]; *chunk = v[3];
    return true;
}

void tune_cache_store(int dims, const int64_t* n, int bc, int dtype, int scheme, int kernel, int depth, int variant,
                      int chunk, double us) {
    const int v[4] = {kernel, depth, variant, chunk};
    store_line(make_key(dims, n, bc, dtype, scheme), v, us);
}

bool tune_cache_lookup_class(const std::string& cls, int* v4) { return lookup_line(device_prefix() + "/" + cls, v4); }

void tune_cache_store_class(const std::string& cls, const int* v4, double us) {
    store_line(device_prefix() + "/" + cls, v4, us);
}

}  // namespace acs
