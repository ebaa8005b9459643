// tune.cu -- on-line autotuner for the tensor-core join's tile configuration.
//
// A configuration is a code: the tile width (128 or 256 columns) plus kTunePair when the tile
// runs on a pair of SMs (tcgen05 cta_group::2, 256-row tiles) or kTuneWide for the 16-warp
// epilogue (which wins when many chunks hold candidates). A tuning key is a shape class:
// (device SMs, padded d, join kind, log2 |R|, log2 |S|). Each kind has its own candidate list;
// the first calls of a class run every candidate once, then the first candidate again (its
// first run is the class's cold call), with CUDA-event timing of the tensor-core kernel. A
// candidate's best kernel milliseconds per 10^9 pairs counts, and from then on the fastest is
// used. The shared-memory plan (stages, resident R-tile slots) follows from the configuration
// and d (tc_plan); top-k's S-split count follows from the grid. Decisions are kept for the
// process and, when the environment variable DL_TUNE_CACHE names a file, loaded from and
// appended to it as lines "key code".
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

namespace dl {

namespace {

constexpr int kMaxCandidates = 4;

struct Entry {
    double ms_per_gpair[kMaxCandidates] = {0.0, 0.0, 0.0, 0.0};   // best trial so far
    int tried = 0;      // trials measured so far
    int chosen = 0;     // 0 until decided
};

std::mutex g_mu;
std::map<std::string, Entry> g_tab;
bool g_loaded = false;

// Candidate configurations of a join kind, fastest-first guess first.
std::vector<int> candidates(int kind)
{
    switch (kind) {
    case kTuneEpsRxS:
    case kTuneEpsSelf:
        return {256, 128, 256 | kTuneWide, 256 | kTunePair};
    case kTuneEpsRxS8:
    case kTuneEpsSelf8:
        return {256, 256 | kTuneWide, 256 | kTunePair};
    case kTuneBatch:
        return {256, 256 | kTuneWide};
    default:   // top-k: single-SM tiles
        return {256, 128, 256 | kTuneWide};
    }
}

int ilog2(int64_t x)
{
    int l = 0;
    while (x > 1) {
        x >>= 1;
        ++l;
    }
    return l;
}

// Batches and top-k calls of a server vary in size from call to call: their query sizes fall
// in classes a factor of four wide, so that a server's shape classes are few and each is tuned
// once (the other kinds: a factor of two).
std::string make_key(int dp, int kind, int64_t nR, int64_t nS)
{
    char buf[96];
    const int lr = (kind == kTuneBatch || kind == kTuneTopk) ? ilog2(nR) / 2 * 2 : ilog2(nR);
    std::snprintf(buf, sizeof buf, "sm%d:dp%d:k%d:r%d:s%d", device_sm_count(), dp, kind, lr, ilog2(nS));
    return buf;
}

void load_locked()
{
    if (g_loaded) return;
    g_loaded = true;
    const char *path = std::getenv("DL_TUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    char key[96];
    int code = 0;
    while (std::fscanf(f, "%95s %d", key, &code) == 2) {
        Entry &e = g_tab[key];
        e.chosen = code;
        e.tried = 1 << 20;
    }
    std::fclose(f);
}

void save_locked(const std::string &key, int code)
{
    const char *path = std::getenv("DL_TUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s %d\n", key.c_str(), code);
    std::fclose(f);
}

// The candidate a class's trial number t runs: each once, then the first again.
int trial_index(int t, int n) { return t < n ? t : 0; }

}  // namespace

int tune_trials(int kind) { return (int)candidates(kind).size() + 1; }

// Configuration code for this shape class; *trial is set when the call measures a candidate.
int tune_pick(int dp, int kind, int64_t nR, int64_t nS, bool *trial)
{
    std::lock_guard<std::mutex> lk(g_mu);
    load_locked();
    Entry &e = g_tab[make_key(dp, kind, nR, nS)];
    if (e.chosen) {
        *trial = false;
        return e.chosen;
    }
    const std::vector<int> c = candidates(kind);
    *trial = true;
    return c[trial_index(e.tried, (int)c.size())];
}

// Record a measured candidate; decides the class once every trial has been timed.
void tune_record(int dp, int kind, int64_t nR, int64_t nS, int code, double kernel_ms, double pairs)
{
    if (!(kernel_ms > 0.0) || !(pairs > 0.0)) return;
    std::lock_guard<std::mutex> lk(g_mu);
    const std::string key = make_key(dp, kind, nR, nS);
    Entry &e = g_tab[key];
    const std::vector<int> c = candidates(kind);
    const int n = (int)c.size();
    if (e.chosen || e.tried > n) return;
    const int i = trial_index(e.tried, n);
    if (c[i] != code) return;
    const double v = kernel_ms / (pairs / 1e9);
    if (e.tried < n || v < e.ms_per_gpair[i]) e.ms_per_gpair[i] = v;
    ++e.tried;
    if (e.tried == n + 1) {
        int best = 0;
        for (int j = 1; j < n; ++j)
            if (e.ms_per_gpair[j] < e.ms_per_gpair[best]) best = j;
        e.chosen = c[best];
        save_locked(key, e.chosen);
    }
}

}  // namespace dl
