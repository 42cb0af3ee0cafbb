// Binomial checkpointing of the adjoint sweep over tape segments: the schedule of restore,
// advance, store, free, tape and adjoint actions that reverses every segment exactly once within
// a number of snapshot slots (Griewank and Walther's bound C(s + r, s)), and the choice of tape
// length for a pool of snapshot slots.  Host only.
#include "lks_engine.h"

using namespace lks::eng;

namespace {

// Number of segments reversible with s free snapshot slots when every segment is advanced at
// most r times: C(s + r, s) (Griewank & Walther's binomial bound), capped.
double binom_beta(int s, int r) {
    double v = 1.0;
    for (int i = 1; i <= s; ++i) {
        v = v * (double)(r + i) / (double)i;
        if (v > 1e15) return 1e15;
    }
    return v;
}

}  // namespace

namespace lks {
namespace eng {

// Reverse segments [a, b) given the state at segment a's start (snapshot or initial state)
// and s free snapshot slots.  The right part is reversed first with one slot fewer; the split
// makes the right part as long as the binomial bound allows, which minimises re-advancing.
void gen_schedule(int a, int b, int s, std::vector<Act>& out) {
    if (b - a == 1) {
        out.push_back({A_RESTORE, a, 0});
        out.push_back({A_TAPE, a, 0});
        out.push_back({A_ADJ, a, 0});
        return;
    }
    if (s <= 0) {
        for (int j = b - 1; j >= a; --j) {
            out.push_back({A_RESTORE, a, 0});
            if (j > a) out.push_back({A_ADVANCE, a, j});
            out.push_back({A_TAPE, j, 0});
            out.push_back({A_ADJ, j, 0});
        }
        return;
    }
    const int L = b - a;
    int r = 1;
    while (binom_beta(s, r) < (double)L) ++r;
    const double right = binom_beta(s - 1, r);
    long long left = (long long)L - (long long)std::min(right, (double)L);
    int m = a + (int)std::max(1LL, left);
    if (m >= b) m = b - 1;
    out.push_back({A_RESTORE, a, 0});
    out.push_back({A_ADVANCE, a, m});
    out.push_back({A_STORE, m, 0});
    gen_schedule(m, b, s - 1, out);
    out.push_back({A_FREE, m, 0});
    gen_schedule(a, m, s, out);
}

// Pick the tape length K and the number of checkpoint slots S for N steps and P pool slots.
void plan_tape(int N, int P, int& K, int& M, int& S) {
    if (P >= N + 1) {
        K = N;
        M = 1;
        S = 0;
        return;
    }
    K = (int)std::ceil(std::sqrt((double)N));
    if (K + 1 > P - 1) K = std::max(1, P / 2 - 1);
    M = (N + K - 1) / K;
    S = P - (K + 1);
    if (S < 0) S = 0;
}

}  // namespace eng
}  // namespace lks

extern "C" int lks_checkpoint_schedule(int n_segments, int free_slots, int* triples, int cap) {
    if (n_segments < 1 || free_slots < 0 || (!triples && cap > 0)) return -1;
    std::vector<Act> acts;
    gen_schedule(0, n_segments, free_slots, acts);
    const int n = (int)std::min<size_t>(acts.size(), (size_t)std::max(cap, 0));
    for (int i = 0; i < n; ++i) {
        triples[3 * i] = acts[i].kind;
        triples[3 * i + 1] = acts[i].a;
        triples[3 * i + 2] = acts[i].b;
    }
    return (int)acts.size();
}
