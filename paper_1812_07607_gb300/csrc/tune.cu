// tune.cu -- on-line autotuner for the tensor-core tile width.
//
// A tuning key is a shape class: (device SMs, padded d, join kind, log2 |R|,
// log2 |S|). The first calls of a class run the candidate tile widths in turn
// (256, 128, 256, 128) with CUDA-event timing of the tensor-core kernel; each
// candidate's best (smallest kernel milliseconds per 10^9 pairs) of its two trials
// counts, so a cold first call does not decide. From then on the faster one is
// used. Decisions are kept for the process and, when the environment variable
// DL_TUNE_CACHE names a file, loaded from and appended to it as lines "key BN".
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>

#include "internal.h"

namespace dl {

namespace {

constexpr int kCandidates[] = {256, 128};
constexpr int kNumCandidates = 2;
constexpr int kRounds = 2;   // trials per candidate
constexpr int kTrials = kNumCandidates * kRounds;

struct Entry {
    double ms_per_gpair[kNumCandidates] = {0.0, 0.0};   // best trial so far
    int tried = 0;      // trials measured so far
    int chosen = 0;     // 0 until decided
};

std::mutex g_mu;
std::map<std::string, Entry> g_tab;
bool g_loaded = false;

int ilog2(int64_t x)
{
    int l = 0;
    while (x > 1) {
        x >>= 1;
        ++l;
    }
    return l;
}

std::string make_key(int dp, int kind, int64_t nR, int64_t nS)
{
    char buf[96];
    std::snprintf(buf, sizeof buf, "sm%d:dp%d:k%d:r%d:s%d", device_sm_count(), dp, kind, ilog2(nR), ilog2(nS));
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
    int bn = 0;
    while (std::fscanf(f, "%95s %d", key, &bn) == 2) {
        Entry &e = g_tab[key];
        e.chosen = bn;
        e.tried = kTrials;
    }
    std::fclose(f);
}

void save_locked(const std::string &key, int bn)
{
    const char *path = std::getenv("DL_TUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s %d\n", key.c_str(), bn);
    std::fclose(f);
}

}  // namespace

// Tile width for this shape class; *trial is set when the call measures a candidate.
int tune_pick(int dp, int kind, int64_t nR, int64_t nS, bool *trial)
{
    std::lock_guard<std::mutex> lk(g_mu);
    load_locked();
    Entry &e = g_tab[make_key(dp, kind, nR, nS)];
    if (e.chosen) {
        *trial = false;
        return e.chosen;
    }
    *trial = true;
    return kCandidates[e.tried % kNumCandidates];
}

// Record a measured candidate; decides the class once every candidate has been timed.
void tune_record(int dp, int kind, int64_t nR, int64_t nS, int bn, double kernel_ms, double pairs)
{
    if (!(kernel_ms > 0.0) || !(pairs > 0.0)) return;
    std::lock_guard<std::mutex> lk(g_mu);
    const std::string key = make_key(dp, kind, nR, nS);
    Entry &e = g_tab[key];
    if (e.chosen || e.tried >= kTrials || kCandidates[e.tried % kNumCandidates] != bn) return;
    const int c = e.tried % kNumCandidates;
    const double v = kernel_ms / (pairs / 1e9);
    if (e.tried < kNumCandidates || v < e.ms_per_gpair[c]) e.ms_per_gpair[c] = v;
    ++e.tried;
    if (e.tried == kTrials) {
        int best = 0;
        for (int i = 1; i < kNumCandidates; ++i)
            if (e.ms_per_gpair[i] < e.ms_per_gpair[best]) best = i;
        e.chosen = kCandidates[best];
        save_locked(key, e.chosen);
    }
}

}  // namespace dl
