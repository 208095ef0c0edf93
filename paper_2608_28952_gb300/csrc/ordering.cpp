// ordering.cpp -- host-side construction of a sweep's pair schedule.
//
// Sec. 3 (item 2): the N(N-1)/2 block pairs I<J are partitioned into groups
// of pairwise disjoint pairs; all transforms of one group are independent and
// run as one parallel step.  Two groupings are offered:
//   * round-robin tournament (the default): block 0 stays in position 0 and
//     blocks 1..N-1 advance one position per step; in step s the block in
//     position j meets the block in position N-1-j.  N-1 steps of N/2 pairs.
//   * Algorithm 3 ("cyclic by anti-diagonals"): group K collects the pairs
//     with (I+J) mod N == K (1-based I, J), for K = 0..N-1.
#include <algorithm>

#include "internal.h"

namespace jac {

int padded_blocks(int n, int b, int ordering)
{
    int N = (n + b - 1) / b;
    if (N < 2) N = 2;  // a single block still needs one (padded) pair
    if (N & 1) N += 1; // every block belongs to exactly one entry of a step
    (void)ordering;
    return N;
}

static void round_robin(int N, Ordering* o)
{
    const int steps = N - 1, half = N / 2;
    // position -> block for the current step, advanced by one slot per step
    std::vector<int> at(N);
    for (int s = 0; s < steps; ++s) {
        at[0] = 0;
        for (int pos = 1; pos < N; ++pos) at[pos] = 1 + (pos - 1 + s) % (N - 1);
        o->step_ptr.push_back((int)o->pairs.size() / 2);
        for (int j = 0; j < half; ++j) {
            int x = at[j], y = at[N - 1 - j];
            o->pairs.push_back(x < y ? x : y);
            o->pairs.push_back(x < y ? y : x);
        }
    }
    o->S = steps;
}

static void anti_diagonal(int N, Ordering* o)
{
    // bucket every 1-based pair by (I+J) mod N, then emit buckets K = 0..N-1
    std::vector<std::vector<int>> bucket(N);
    for (int I = 1; I < N; ++I)
        for (int J = I + 1; J <= N; ++J) {
            bucket[(I + J) % N].push_back(I - 1);
            bucket[(I + J) % N].push_back(J - 1);
        }
    for (int K = 0; K < N; ++K) {
        o->step_ptr.push_back((int)o->pairs.size() / 2);
        o->pairs.insert(o->pairs.end(), bucket[K].begin(), bucket[K].end());
    }
    o->S = N;
}

bool make_ordering(int kind, int N, Ordering* o)
{
    *o = Ordering();
    o->N = N;
    if (N < 2) return false;
    if (kind == JACOBI_ORDER_ROUND_ROBIN) {
        if (N & 1) return false;
        round_robin(N, o);
    } else if (kind == JACOBI_ORDER_ANTI_DIAGONAL) {
        anti_diagonal(N, o);
    } else {
        return false;
    }
    o->step_ptr.push_back((int)o->pairs.size() / 2);
    for (int s = 0; s < o->S; ++s) {
        int c = o->step_ptr[s + 1] - o->step_ptr[s];
        if (c > o->max_pairs) o->max_pairs = c;
    }
    // device schedule: N/2 entries per step (N even), frozen entry for the
    // blocks a step leaves out
    if ((N & 1) == 0) {
        o->dev_per_step = N / 2;
        std::vector<char> used(N);
        for (int s = 0; s < o->S; ++s) {
            std::fill(used.begin(), used.end(), 0);
            for (int e = o->step_ptr[s]; e < o->step_ptr[s + 1]; ++e) {
                o->dev_pairs.push_back(o->pairs[2 * e]);
                o->dev_pairs.push_back(o->pairs[2 * e + 1]);
                used[o->pairs[2 * e]] = used[o->pairs[2 * e + 1]] = 1;
            }
            std::vector<int> left;
            for (int x = 0; x < N; ++x)
                if (!used[x]) left.push_back(x);
            for (size_t i = 0; i + 1 < left.size(); i += 2) {
                o->dev_pairs.push_back(-1 - left[i]);
                o->dev_pairs.push_back(-1 - left[i + 1]);
            }
        }
        o->max_pairs = o->dev_per_step;
    }
    return true;
}

}  // namespace jac

// Exported for the host-logic tests (no GPU needed): the schedule as
// 0-based pairs.  pairs needs N*(N-1) ints, step_ptr N+1.  Returns S or <0.
extern "C" int jacobi_ordering_table(int kind, int N, int* pairs, int* step_ptr)
{
    jac::Ordering o;
    if (!jac::make_ordering(kind, N, &o)) return -1;
    for (size_t i = 0; i < o.pairs.size(); ++i) pairs[i] = o.pairs[i];
    for (int s = 0; s <= o.S; ++s) step_ptr[s] = o.step_ptr[s];
    return o.S;
}
