// hv_schedule.cpp -- binomial wavefield checkpointing for the adjoint sweep.
//
// The Hessian apply and the gradient run the wave equation forward and its
// adjoint backward in time (paper section 3: each H_d v needs the forward
// field while the adjoint field is stepped backward).  With a budget of
// `slots` stored states per shot, the forward field is recomputed from
// snapshots.  State x_j = (u^j, u^{j-1}); x_0 = 0 is free; the adjoint of step
// n needs u^n, which is x_n's first or x_{n+1}'s second level.
//
// The first forward sweep (which must run anyway for the Born data) stores
// snapshots; the reversal then restores snapshots and recomputes.  The number
// of recomputed steps is minimised exactly:
//   * reversing a segment of L states with its start stored and f free slots
//     costs A(L, f) = t L - binom(f + 2 + t - 1, t - 1) with t the smallest
//     integer such that binom(f + 1 + t, t) >= L (Griewank 1992, binomial
//     checkpointing); the split point is the argmin of m + A(L-m, f-1) + A(m, f);
//   * the first-sweep snapshot positions minimise
//     W(n, f) = min(A(n-1, f), min_m W(n-m, f-1) + A(m, f))
//     (the sweep ends holding x_nt, so the adjoint of step nt-1 is free).
#include "hv_internal.h"

#include <algorithm>
#include <limits>

namespace hvi {

namespace {

// binom(s + t, t), saturating at a large value.
long long beta(int s, int t)
{
    if (t < 0) return 0;
    long double v = 1.0L;
    for (int i = 1; i <= t; ++i) {
        v = v * (long double)(s + i) / (long double)i;
        if (v > 4.0e18L) return (long long)4e18;
    }
    return (long long)(v + 0.5L);
}

}  // namespace

long long seg_cost(long long L, int f)
{
    if (L <= 1) return 0;
    if (f <= 0) return L * (L - 1) / 2;
    int S = f + 1;
    int t = 0;
    while (beta(S, t) < L) ++t;
    return t * L - beta(S + 1, t - 1);
}

namespace {

struct Emitter {
    std::vector<Action> &out;
    const std::vector<std::vector<long long>> &A;   // A[f][L] = seg_cost(L, f)
    std::vector<int> free_slots;
    long long advances = 0;
    int cur_state = -1;      // state index currently held (-1: unknown)

    void emit(int op, int a0, int a1) { out.push_back(Action{op, a0, a1}); }

    void restore(int slot, int state)
    {
        emit(ACT_RESTORE, slot, state);
        cur_state = state;
    }
    void advance(int n)
    {
        for (int i = 0; i < n; ++i) emit(ACT_ADVANCE, cur_state + i, 0);
        cur_state += n;
        advances += n;
    }

    int best_split(long long L, int f)
    {
        long long best = std::numeric_limits<long long>::max();
        int arg = 1;
        for (long long m = 1; m < L; ++m) {
            long long c = m + A[f - 1][L - m] + A[f][m];
            if (c < best) { best = c; arg = (int)m; }
        }
        return arg;
    }

    // Reverse adjoint steps p+L-1 .. p with x_p stored in `slot` (-1: zero state).
    void reverse_segment(int p, long long L, int slot)
    {
        int f = (int)free_slots.size();
        if (L <= 0) return;
        if (L == 1) {
            if (cur_state != p) restore(slot, p);
            emit(ACT_ADJOINT, p, 0);
            return;
        }
        if (f == 0) {
            for (long long i = L - 1; i >= 0; --i) {
                restore(slot, p);
                advance((int)i);
                emit(ACT_ADJOINT, p + (int)i, 0);
            }
            return;
        }
        int m = best_split(L, f);
        restore(slot, p);
        advance(m);
        int ns = free_slots.back();
        free_slots.pop_back();
        emit(ACT_SAVE, ns, p + m);
        reverse_segment(p + m, L - m, ns);
        free_slots.push_back(ns);
        reverse_segment(p, m, slot);
    }
};

}  // namespace

int build_schedule(int nt, int slots, std::vector<Action> &out, long long *n_advances)
{
    out.clear();
    if (nt < 1 || slots < 0) return -1;
    if (slots > nt) slots = nt;
    // W table: W[f][n], choice[f][n] (0 = no further first-sweep snapshot, else m).
    std::vector<std::vector<long long>> W(slots + 1, std::vector<long long>(nt + 1, 0));
    std::vector<std::vector<int>> choice(slots + 1, std::vector<int>(nt + 1, 0));
    std::vector<std::vector<long long>> A(slots + 1, std::vector<long long>(nt + 1, 0));
    for (int f = 0; f <= slots; ++f)
        for (int L = 0; L <= nt; ++L) A[f][L] = seg_cost(L, f);
    for (int f = 0; f <= slots; ++f) {
        for (int n = 1; n <= nt; ++n) {
            long long best = A[f][n - 1];
            int arg = 0;
            if (f >= 1)
                for (int m = 1; m < n; ++m) {
                    long long c = W[f - 1][n - m] + A[f][m];
                    if (c < best) { best = c; arg = m; }
                }
            W[f][n] = best;
            choice[f][n] = arg;
        }
    }
    // First-sweep snapshot positions.
    std::vector<int> pos;
    {
        int f = slots, n = nt, p = 0;
        while (n > 1 && f >= 1 && choice[f][n] != 0) {
            int m = choice[f][n];
            p += m;
            pos.push_back(p);
            n -= m;
            --f;
        }
    }
    // First sweep: forward steps with saves into slots 0..k-1.
    size_t k = 0;
    for (int n = 0; n < nt; ++n) {
        out.push_back(Action{ACT_FORWARD, n, 0});
        if (k < pos.size() && pos[k] == n + 1) {
            out.push_back(Action{ACT_SAVE, (int)k, n + 1});
            ++k;
        }
    }
    Emitter E{out, A};
    E.cur_state = nt;   // the sweep ends holding x_nt (u^nt, u^{nt-1})
    for (int s = slots - 1; s >= (int)pos.size(); --s) E.free_slots.push_back(s);
    // Tail: adjoint nt-1 from x_nt, then the segment [p_k, nt-1).
    out.push_back(Action{ACT_ADJOINT, nt - 1, 0});
    int pk = pos.empty() ? 0 : pos.back();
    int slot_k = pos.empty() ? -1 : (int)pos.size() - 1;
    E.reverse_segment(pk, (long long)(nt - 1 - pk), slot_k);
    // Earlier segments, each after the later ones freed their slots.
    for (int j = (int)pos.size() - 1; j >= 0; --j) {
        E.free_slots.push_back(j);   // slot j held p_{j+1}, whose segment is done
        int start = (j == 0) ? 0 : pos[j - 1];
        int sslot = (j == 0) ? -1 : j - 1;
        // segment [start, pos[j]) with f = free slots
        E.reverse_segment(start, (long long)(pos[j] - start), sslot);
    }
    if (n_advances) *n_advances = E.advances;
    return 0;
}

}  // namespace hvi

extern "C" int hv_checkpoint_schedule(int nt, int slots, int *actions, int max_actions, int *n_actions,
                                      long long *n_advances)
{
    std::vector<hvi::Action> acts;
    long long adv = 0;
    if (nt < 1 || slots < 0) return hvi::fail(HV_EINVAL, "hv_checkpoint_schedule: nt >= 1 and slots >= 0 required");
    hvi::build_schedule(nt, slots, acts, &adv);
    if (n_actions) *n_actions = (int)acts.size();
    if (n_advances) *n_advances = adv;
    if (actions) {
        if ((int)acts.size() > max_actions)
            return hvi::fail(HV_ENOMEM, "hv_checkpoint_schedule: %d actions do not fit in %d", (int)acts.size(),
                             max_actions);
        for (size_t i = 0; i < acts.size(); ++i) {
            actions[3 * i + 0] = acts[i].op;
            actions[3 * i + 1] = acts[i].a0;
            actions[3 * i + 2] = acts[i].a1;
        }
    }
    return hvi::ok();
}
