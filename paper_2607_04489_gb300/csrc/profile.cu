// Per-launch timing of the join pipeline (eiger_profile / eiger_profile_read).
#include <cstring>
#include <vector>

#include "eiger.h"
#include "kernels.cuh"

namespace eiger {

namespace {

struct Rec {
    char name[32];
    double bytes;
    double per_match;
    int launches;
    cudaEvent_t ev[2];
};

struct ProfState {
    bool enabled = false;
    int used = 0;
    unsigned long long matches = 0;
    std::vector<Rec> recs;
    ~ProfState() {
        for (Rec& r : recs) {
            cudaEventDestroy(r.ev[0]);
            cudaEventDestroy(r.ev[1]);
        }
    }
};

thread_local ProfState g_prof;

}  // namespace

ProfScope::ProfScope(const char* name, double bytes, cudaStream_t s, double per_match, int launches)
    : stream(s), slot(-1) {
    if (!g_prof.enabled) return;
    if (g_prof.used == (int)g_prof.recs.size()) {
        Rec r{};
        if (cudaEventCreate(&r.ev[0]) != cudaSuccess || cudaEventCreate(&r.ev[1]) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        g_prof.recs.push_back(r);
    }
    slot = g_prof.used++;
    Rec& r = g_prof.recs[slot];
    std::strncpy(r.name, name, sizeof r.name - 1);
    r.name[sizeof r.name - 1] = 0;
    r.bytes = bytes;
    r.per_match = per_match;
    r.launches = launches;
    cudaEventRecord(r.ev[0], stream);
}

ProfScope::~ProfScope() {
    if (slot >= 0) cudaEventRecord(g_prof.recs[slot].ev[1], stream);
}

void prof_reset() {
    g_prof.used = 0;
    g_prof.matches = 0;
}
void prof_set_matches(unsigned long long m) { g_prof.matches = m; }

double match_bytes(const JoinOut& out) {
    if (out.aggregate) return 2.0 * out.b.bytes[0];  // both payloads read per match
    double b = 0;
    if (out.bidx) b += out.b.rowmap ? 8 : 4;  // (rowmap read +) index written
    if (out.pidx) b += out.p.rowmap ? 8 : 4;
    for (int c = 0; c < out.b.n; ++c) b += 2.0 * out.b.bytes[c];  // gathered and written
    for (int c = 0; c < out.p.n; ++c) b += 2.0 * out.p.bytes[c];
    return b;
}
int prof_count() { return g_prof.used; }

bool prof_enabled() { return g_prof.enabled; }

bool prof_set_enabled(bool on) {
    const bool was = g_prof.enabled;
    g_prof.enabled = on;
    return was;
}

}  // namespace eiger

using namespace eiger;

extern "C" {

eiger_status eiger_profile(int enable) {
    g_prof.enabled = enable != 0;
    g_prof.used = 0;
    return EIGER_OK;
}

int eiger_profile_read(eiger_stage_t* out, int max_stages) {
    int n = g_prof.used;
    if (!out) return n;
    if (n > max_stages) n = max_stages;
    for (int i = 0; i < n; ++i) {
        Rec& r = g_prof.recs[i];
        std::memcpy(out[i].name, r.name, sizeof out[i].name);
        out[i].bytes = r.bytes + r.per_match * (double)g_prof.matches;
        out[i].launches = r.launches;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.ev[0], r.ev[1]) != cudaSuccess) {
            cudaGetLastError();
            ms = -1.f;
        }
        out[i].ms = ms;
    }
    return n;
}

}  // extern "C"
