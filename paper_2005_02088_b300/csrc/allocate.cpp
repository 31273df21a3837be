// camelot_allocate: the two contention-aware allocation policies.
//
// Peak-load policy (Eq. 1) and low-load resource policy (Eq. 3) over the
// allocation vector V = [N_1..N_n, p_1..p_n] (end of Sec. 7.3) and a candidate
// batch size (Eq. 3 makes the batch a variable).  The exhaustive solver walks
// every stage's (instances, quota level) pairs depth first, pruning a branch
// as soon as a partial sum already breaks a budget (every table entry is
// non-negative, so partial sums only grow).  The annealing solver is the
// paper's: random one-step moves of V, infeasible moves dropped, worse moves
// accepted with a probability that decays with a geometric temperature,
// from several starting states.  Host code only.
#include <algorithm>
#include <deque>
#include <queue>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/camelot.h"

void camelot_internal_set_error(const char* msg);   // runtime.cpp: camelot_last_error's slot

namespace {

camelot_status set_err(camelot_status s, const char* msg) {
    camelot_internal_set_error(msg);
    return s;
}

struct Problem {
    int n, L, nb, unit, S, I, policy, maxN;
    const double *f, *bw, *d, *mem;
    double BW, F, qos, load;
    const double* hb;   // host-link demand per instance (nullptr: no host-link constraint)
    double HB;          // host-link budget
    size_t k(int b, int i, int l) const { return ((size_t)b * n + i) * L + l; }
};

// A candidate and its ordering key.
struct Cand {
    bool ok = false;
    int b = 0;
    std::vector<int> N, l;
    double thr = 0.0;
    int sms = 0;
};

// Is (thr, sms, b, N, l) strictly better than `best`?
bool better(const Problem& P, double thr, int sms, int b, const int* N, const int* l,
            const Cand& best) {
    if (!best.ok) return true;
    if (P.policy == CAMELOT_POLICY_MAX_PEAK) {
        if (thr != best.thr) return thr > best.thr;
        if (sms != best.sms) return sms < best.sms;
    } else {
        if (sms != best.sms) return sms < best.sms;
        if (thr != best.thr) return thr > best.thr;
    }
    if (b != best.b) return b < best.b;
    for (int i = 0; i < P.n; ++i)
        if (N[i] != best.N[i]) return N[i] < best.N[i];
    for (int i = 0; i < P.n; ++i)
        if (l[i] != best.l[i]) return l[i] < best.l[i];
    return false;
}

// Full evaluation of one state, summing in stage order.
bool feasible(const Problem& P, int b, const int* N, const int* l, double* thr, int* sms) {
    long long sm = 0, inst = 0;
    double bws = 0.0, mems = 0.0, dur = 0.0, tmin = INFINITY, hbs = 0.0;
    for (int i = 0; i < P.n; ++i) {
        if (N[i] < 1 || N[i] > P.maxN || l[i] < 0 || l[i] >= P.L) return false;
        const size_t k = P.k(b, i, l[i]);
        sm += (long long)N[i] * (l[i] + 1) * P.unit;
        inst += N[i];
        bws += N[i] * P.bw[k];
        mems += N[i] * P.mem[(size_t)b * P.n + i];
        dur += P.d[k];
        if (P.hb) hbs += N[i] * P.hb[k];
        tmin = std::min(tmin, N[i] * P.f[k]);
    }
    if (sm > P.S || inst > P.I || bws > P.BW || mems > P.F || dur > P.qos) return false;
    if (P.hb && hbs > P.HB) return false;
    if (P.policy == CAMELOT_POLICY_MIN_SM && tmin < P.load) return false;
    *thr = tmin;
    *sms = (int)sm;
    return true;
}

struct Dfs {
    const Problem& P;
    int b;
    std::vector<int> N, l;
    Cand& best;
    void run(int i, long long sm, long long inst, double bws, double mems, double dur, double hbs) {
        if (i == P.n) {
            double thr;
            int sms;
            if (feasible(P, b, N.data(), l.data(), &thr, &sms) &&
                better(P, thr, sms, b, N.data(), l.data(), best)) {
                best.ok = true;
                best.b = b;
                best.N = N;
                best.l = l;
                best.thr = thr;
                best.sms = sms;
            }
            return;
        }
        for (int n = 1; n <= P.maxN; ++n) {
            if (inst + n > P.I) break;
            const double m2 = mems + n * P.mem[(size_t)b * P.n + i];
            if (m2 > P.F) break;
            for (int lv = 0; lv < P.L; ++lv) {
                const long long sm2 = sm + (long long)n * (lv + 1) * P.unit;
                if (sm2 > P.S) break;
                const size_t k = P.k(b, i, lv);
                const double bw2 = bws + n * P.bw[k];
                const double d2 = dur + P.d[k];
                const double h2 = P.hb ? hbs + n * P.hb[k] : 0.0;
                if (bw2 > P.BW || d2 > P.qos || (P.hb && h2 > P.HB)) continue;
                N[i] = n;
                l[i] = lv;
                run(i + 1, sm2, inst + n, bw2, m2, d2, h2);
            }
        }
    }
};

uint64_t sm64(uint64_t* s) {   // SplitMix64 (Steele, Lea & Flood 2014)
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void anneal(const Problem& P, int iters, double T0, double alpha, uint64_t seed, Cand& best) {
    uint64_t rs = seed ^ 0x5851F42D4C957F2Dull;
    std::vector<int> N(P.n), l(P.n), N2, l2;
    // Four walks per batch size: the first from N_i = 1 at the lowest level, the
    // others from random feasible states, since single-step moves cannot cross
    // an infeasible gap in V.
    for (int walk = 0; walk < 4 * P.nb; ++walk) {
        const int b = walk / 4;
        std::fill(N.begin(), N.end(), 1);
        std::fill(l.begin(), l.end(), 0);
        double thr = 0;
        int sms = 0;
        bool have = (walk % 4 == 0) && feasible(P, b, N.data(), l.data(), &thr, &sms);
        for (int t = 0; t < 20000 && !have; ++t) {
            for (int i = 0; i < P.n; ++i) {
                N[i] = 1 + (int)(sm64(&rs) % (uint64_t)P.maxN);
                l[i] = (int)(sm64(&rs) % (uint64_t)P.L);
            }
            have = feasible(P, b, N.data(), l.data(), &thr, &sms);
        }
        if (!have) continue;
        if (better(P, thr, sms, b, N.data(), l.data(), best))
            best = Cand{true, b, N, l, thr, sms};
        const double scale = P.policy == CAMELOT_POLICY_MAX_PEAK ? std::max(thr, 1e-300) : (double)P.S;
        double T = T0;
        for (int it = 0; it < iters; ++it, T *= alpha) {
            N2 = N;
            l2 = l;
            const uint64_t r = sm64(&rs);
            const int coord = (int)((r >> 1) % (uint64_t)(2 * P.n));
            const int step = (r & 1) ? 1 : -1;
            if (coord < P.n) N2[coord] += step; else l2[coord - P.n] += step;
            double thr2;
            int sms2;
            if (!feasible(P, b, N2.data(), l2.data(), &thr2, &sms2)) continue;
            const double gain = P.policy == CAMELOT_POLICY_MAX_PEAK ? (thr2 - thr) / scale
                                                                     : (double)(sms - sms2) / scale;
            const double u = (sm64(&rs) >> 11) * 0x1.0p-53;
            if (gain > 0 || (T > 0 && u < std::exp(gain / T))) {
                N.swap(N2);
                l.swap(l2);
                thr = thr2;
                sms = sms2;
                if (better(P, thr, sms, b, N.data(), l.data(), best))
                    best = Cand{true, b, N, l, thr, sms};
            }
        }
    }
}

}  // namespace

extern "C" camelot_status camelot_allocate(const camelot_profile* prof, camelot_policy policy,
                                           const camelot_constraints* c, camelot_alloc* out,
                                           double* objective) {
    if (!prof || !c || !out) return set_err(CAMELOT_EINVAL, "null argument");
    if (policy != CAMELOT_POLICY_MAX_PEAK && policy != CAMELOT_POLICY_MIN_SM)
        return set_err(CAMELOT_EINVAL, "unknown policy");
    if (prof->n_stages < 1 || prof->n_stages > CAMELOT_MAX_STAGES || prof->n_levels < 1 ||
        prof->n_batches < 1 || prof->unit < 1)
        return set_err(CAMELOT_EINVAL, "bad profile sizes");
    if (!prof->thr_qps || !prof->bw_gbs || !prof->dur_s || !prof->mem_bytes || !prof->batch_sizes)
        return set_err(CAMELOT_EINVAL, "profile table missing");
    if (c->total_sms < 1 || c->max_instances < 1) return set_err(CAMELOT_EINVAL, "bad constraints");
    const size_t cells = (size_t)prof->n_batches * prof->n_stages * prof->n_levels;
    for (size_t i = 0; i < cells; ++i)
        if (!(prof->thr_qps[i] >= 0) || !(prof->bw_gbs[i] >= 0) || !(prof->dur_s[i] >= 0) ||
            (prof->host_gbs && !(prof->host_gbs[i] >= 0)))
            return set_err(CAMELOT_EINVAL, "profile entries must be finite and >= 0");
    if (!(c->host_gbs >= 0)) return set_err(CAMELOT_EINVAL, "host_gbs must be >= 0");
    for (size_t i = 0; i < (size_t)prof->n_batches * prof->n_stages; ++i)
        if (!(prof->mem_bytes[i] >= 0)) return set_err(CAMELOT_EINVAL, "memory entries must be >= 0");
    Problem P{prof->n_stages, prof->n_levels, prof->n_batches, prof->unit, c->total_sms,
              c->max_instances, (int)policy,
              std::max(1, std::min(c->max_instances, c->total_sms / prof->unit)),
              prof->thr_qps, prof->bw_gbs, prof->dur_s, prof->mem_bytes,
              c->bw_gbs, c->mem_bytes, c->qos_s, c->load_qps,
              (prof->host_gbs && c->host_gbs > 0) ? prof->host_gbs : nullptr, c->host_gbs};
    Cand best;
    if (c->solver == CAMELOT_SOLVER_EXHAUSTIVE) {
        for (int b = 0; b < P.nb; ++b) {
            Dfs dfs{P, b, std::vector<int>(P.n, 1), std::vector<int>(P.n, 0), best};
            dfs.run(0, 0, 0, 0.0, 0.0, 0.0, 0.0);
        }
    } else if (c->solver == CAMELOT_SOLVER_ANNEAL) {
        anneal(P, c->anneal_iters > 0 ? c->anneal_iters : 5000,
               c->anneal_t0 > 0 ? c->anneal_t0 : 1.0, c->anneal_alpha > 0 ? c->anneal_alpha : 0.995,
               c->seed, best);
    } else {
        return set_err(CAMELOT_EINVAL, "unknown solver");
    }
    if (!best.ok) return set_err(CAMELOT_EINFEASIBLE, "no allocation satisfies the constraints");
    memset(out, 0, sizeof *out);
    out->n_stages = P.n;
    for (int i = 0; i < P.n; ++i) {
        out->instances[i] = best.N[i];
        out->sm_quota[i] = (best.l[i] + 1) * P.unit;
    }
    out->batch = prof->batch_sizes[best.b];
    if (objective) *objective = policy == CAMELOT_POLICY_MAX_PEAK ? best.thr : (double)best.sms;
    return CAMELOT_OK;
}

namespace {
// Checks a profile against an allocation and returns each stage's quota level.
camelot_status profile_levels(const camelot_profile* prof, const camelot_alloc* alloc, int* level) {
    if (!prof || !alloc || !prof->batch_sizes || !prof->dur_s) return set_err(CAMELOT_EINVAL, "null argument");
    const int n = prof->n_stages, L = prof->n_levels, nb = prof->n_batches, unit = prof->unit;
    if (n < 1 || n > CAMELOT_MAX_STAGES || L < 1 || nb < 1 || unit < 1 || alloc->n_stages != n)
        return set_err(CAMELOT_EINVAL, "profile and allocation shapes disagree");
    for (int j = 0; j < nb; ++j)
        if (prof->batch_sizes[j] < 1 || (j > 0 && prof->batch_sizes[j] <= prof->batch_sizes[j - 1]))
            return set_err(CAMELOT_EINVAL, "batch_sizes must be positive and increasing");
    for (int i = 0; i < n; ++i) {
        const int q = alloc->sm_quota[i];
        if (q < unit || q % unit != 0 || q / unit > L)
            return set_err(CAMELOT_EINVAL, "an SM quota is not a level of the profile");
        level[i] = q / unit - 1;
    }
    return CAMELOT_OK;
}

// Duration of a b-query batch of stage i at its level: linear between the
// profiled batch sizes, the smallest one's below them, in proportion to b above.
double stage_duration(const camelot_profile* prof, const int* level, int i, int b) {
    const int n = prof->n_stages, L = prof->n_levels, nb = prof->n_batches;
    const int* bs = prof->batch_sizes;
    auto dur = [&](int j) { return prof->dur_s[((size_t)j * n + i) * L + level[i]]; };
    if (b <= bs[0]) return dur(0);
    if (b >= bs[nb - 1]) return dur(nb - 1) * (double)b / (double)bs[nb - 1];
    int j = 0;
    while (bs[j + 1] < b) ++j;
    const double f = (double)(b - bs[j]) / (double)(bs[j + 1] - bs[j]);
    return dur(j) + f * (dur(j + 1) - dur(j));
}
}  // namespace

extern "C" camelot_status camelot_trigger_latency(const camelot_profile* prof, const camelot_alloc* alloc,
                                                  int64_t* out_ns) {
    if (!out_ns) return set_err(CAMELOT_EINVAL, "null argument");
    int level[CAMELOT_MAX_STAGES];
    const camelot_status st = profile_levels(prof, alloc, level);
    if (st != CAMELOT_OK) return st;
    for (int b = 1; b <= 32; ++b) {
        double t = 0.0;
        for (int i = 0; i < prof->n_stages; ++i) {
            const double d = stage_duration(prof, level, i, b);
            if (!(d >= 0.0)) return set_err(CAMELOT_EINVAL, "negative or NaN duration in the profile");
            t += d;
        }
        out_ns[b - 1] = (int64_t)std::llround(t * 1e9);
    }
    return CAMELOT_OK;
}

extern "C" camelot_status camelot_profile_add_handover(const camelot_profile* prof, const double* handover_s,
                                                       double* thr, double* bw, double* dur) {
    if (!prof || !handover_s || !thr || !bw || !dur || !prof->thr_qps || !prof->bw_gbs || !prof->dur_s ||
        !prof->batch_sizes)
        return set_err(CAMELOT_EINVAL, "null argument");
    const int n = prof->n_stages, L = prof->n_levels, nb = prof->n_batches;
    if (n < 1 || L < 1 || nb < 1) return set_err(CAMELOT_EINVAL, "empty profile");
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(handover_s[i])) return set_err(CAMELOT_EINVAL, "hand-over times must be finite");
    for (int b = 0; b < nb; ++b)
        for (int i = 0; i < n; ++i)
            for (int l = 0; l < L; ++l) {
                const size_t k = ((size_t)b * n + i) * L + l;
                const double d = prof->dur_s[k];
                if (!(d > 0.0)) return set_err(CAMELOT_EINVAL, "durations must be positive");
                const double bytes = prof->bw_gbs[k] * d;     // GB moved by one batch
                const double d2 = d + handover_s[i];
                if (!(d2 > 0.0)) return set_err(CAMELOT_EINVAL, "a corrected duration is not positive");
                dur[k] = d2;
                thr[k] = (double)prof->batch_sizes[b] / d2;
                bw[k] = bytes / d2;
            }
    return CAMELOT_OK;
}

// ---------------------------------------------------------------------------
// Pipeline simulation on the profile: Poisson arrivals, the batch trigger and
// N_i instances per stage, each batch's service time the profiled duration of
// its size at the stage's quota plus the stage's hand-over time.
// ---------------------------------------------------------------------------
namespace {
struct SimBatch {
    uint64_t first;
    int n;
};
struct SimEvent {
    double t;
    int stage;
    uint64_t batch;
    bool operator<(const SimEvent& o) const { return t > o.t || (t == o.t && stage < o.stage); }
};
}  // namespace

extern "C" camelot_status camelot_simulate_profile(const camelot_profile* prof, const camelot_alloc* alloc,
                                                   const double* handover_s, double max_wait_s, double rate_qps,
                                                   uint32_t n_queries, uint64_t seed, double* p50_s,
                                                   double* p99_s, double* thr_qps) {
    if (!p50_s || !p99_s || !thr_qps) return set_err(CAMELOT_EINVAL, "null argument");
    int level[CAMELOT_MAX_STAGES];
    const camelot_status st = profile_levels(prof, alloc, level);
    if (st != CAMELOT_OK) return st;
    const int n = prof->n_stages, B = alloc->batch;
    if (B < 1 || B > 32 || !(rate_qps > 0.0) || n_queries < 10 || !(max_wait_s >= 0.0))
        return set_err(CAMELOT_EINVAL, "batch 1..32, rate > 0, >= 10 queries, max_wait >= 0 required");
    std::vector<std::vector<double>> svc(n, std::vector<double>(B + 1, 0.0));
    for (int i = 0; i < n; ++i) {
        if (alloc->instances[i] < 1) return set_err(CAMELOT_EINVAL, "instances must be >= 1");
        const double h = handover_s ? handover_s[i] : 0.0;
        if (!std::isfinite(h)) return set_err(CAMELOT_EINVAL, "hand-over times must be finite");
        for (int b = 1; b <= B; ++b) {
            svc[i][b] = stage_duration(prof, level, i, b) + h;
            if (!(svc[i][b] > 0.0)) return set_err(CAMELOT_EINVAL, "a corrected duration is not positive");
        }
    }
    // arrivals: exponential gaps from a SplitMix64 stream
    std::vector<double> arr(n_queries), done(n_queries, 0.0);
    uint64_t x = seed;
    double t = 0.0;
    for (uint32_t q = 0; q < n_queries; ++q) {
        x += 0x9E3779B97F4A7C15ull;
        uint64_t z = x;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        const double u = ((double)(z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        t += -std::log(u) / rate_qps;
        arr[q] = t;
    }
    std::vector<SimBatch> batches;
    std::vector<std::deque<uint64_t>> queue(n);   // batches waiting for stage i (i >= 1)
    std::vector<int> free_inst(alloc->instances, alloc->instances + n);
    std::priority_queue<SimEvent> ev;
    uint64_t next = 0, taken = 0, completed = 0;   // next arrival; first query not yet batched
    double now = 0.0;
    while (completed < n_queries) {
        // start whatever can start now: later stages first, then the trigger
        for (int i = n - 1; i >= 1; --i)
            while (free_inst[i] > 0 && !queue[i].empty()) {
                const uint64_t bi = queue[i].front();
                queue[i].pop_front();
                --free_inst[i];
                ev.push({now + svc[i][batches[bi].n], i, bi});
            }
        while (next < n_queries && arr[next] <= now) ++next;
        while (free_inst[0] > 0 && taken < next) {
            const uint64_t waiting = next - taken;
            const bool full = waiting >= (uint64_t)B;
            if (!full && now < arr[taken] + max_wait_s) break;
            const int b = (int)std::min<uint64_t>(waiting, (uint64_t)B);
            batches.push_back({taken, b});
            taken += b;
            --free_inst[0];
            ev.push({now + svc[0][b], 0, batches.size() - 1});
        }
        // the next moment something changes
        double t_next = INFINITY;
        if (!ev.empty()) t_next = ev.top().t;
        if (next < n_queries) t_next = std::min(t_next, arr[next]);
        if (taken < next && free_inst[0] > 0) t_next = std::min(t_next, arr[taken] + max_wait_s);
        if (!(t_next < INFINITY)) return set_err(CAMELOT_EINVAL, "simulation stalled");
        now = std::max(now, t_next);
        while (!ev.empty() && ev.top().t <= now) {
            const SimEvent e = ev.top();
            ev.pop();
            ++free_inst[e.stage];
            if (e.stage + 1 < n) {
                queue[e.stage + 1].push_back(e.batch);
            } else {
                const SimBatch& sb = batches[e.batch];
                for (int k = 0; k < sb.n; ++k) done[sb.first + k] = e.t;
                completed += sb.n;
            }
        }
    }
    // latencies after the first 10 % (warm-up)
    const uint32_t skip = n_queries / 10;
    std::vector<double> lat;
    lat.reserve(n_queries - skip);
    for (uint32_t q = skip; q < n_queries; ++q) lat.push_back(done[q] - arr[q]);
    std::sort(lat.begin(), lat.end());
    auto pct = [&](double p) {
        const double pos = p * (double)(lat.size() - 1);
        const size_t lo = (size_t)pos;
        const size_t hi = std::min(lo + 1, lat.size() - 1);
        return lat[lo] + (pos - (double)lo) * (lat[hi] - lat[lo]);
    };
    *p50_s = pct(0.50);
    *p99_s = pct(0.99);
    // completions per second after the first 10 % of them
    std::vector<double> fin(done);
    std::sort(fin.begin(), fin.end());
    *thr_qps = (double)(n_queries - skip) / (fin[n_queries - 1] - fin[skip > 0 ? skip - 1 : 0]);
    return CAMELOT_OK;
}
