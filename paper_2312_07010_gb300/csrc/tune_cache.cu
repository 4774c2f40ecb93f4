// tune_cache.cu -- the autotuner's cache: one line per problem class,
//   <key> <kernel> <depth> <variant> <chunk> <microseconds per step>
// where <key> names the device (name and SM count), dims, n, bc, dtype and scheme.
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
    const std::string path = cache_path();
    if (path.empty()) return false;
    const std::string key = make_key(dims, n, bc, dtype, scheme);
    std::lock_guard<std::mutex> lock(g_mu);
    FILE* f = std::fopen(path.c_str(), "r");
    if (!f) return false;
    char line[512], k[300];
    bool found = false;
    while (std::fgets(line, sizeof(line), f)) {
        int a, b, v, ch;
        double us;
        if (std::sscanf(line, "%299s %d %d %d %d %lf", k, &a, &b, &v, &ch, &us) == 6 && key == k) {
            *kernel = a; *depth = b; *variant = v; *chunk = ch;
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

void tune_cache_store(int dims, const int64_t* n, int bc, int dtype, int scheme, int kernel, int depth, int variant,
                      int chunk, double us) {
    const std::string path = cache_path();
    if (path.empty()) return;
    const std::string key = make_key(dims, n, bc, dtype, scheme);
    std::lock_guard<std::mutex> lock(g_mu);
    FILE* f = std::fopen(path.c_str(), "a");
    if (!f) {
        // create the directory of the default location once
        const std::string dir = path.substr(0, path.find_last_of('/'));
        // create the missing directories of the path, one component at a time
        for (size_t i = 1; i <= dir.size(); ++i)
            if (i == dir.size() || dir[i] == '/') (void)mkdir(dir.substr(0, i).c_str(), 0755);
        f = std::fopen(path.c_str(), "a");
        if (!f) return;
    }
    std::fprintf(f, "%s %d %d %d %d %.3f\n", key.c_str(), kernel, depth, variant, chunk, us);
    std::fclose(f);
}

}  // namespace acs
