// Host side of the sector basis: occupation strings in rank order and the
// nearest-neighbour hopping tables of the 1D chain (Eq. 9).
//
// Sign rule.  With the Jordan-Wigner order "all up orbitals, then all down
// orbitals", a hop of one spin species between the neighbouring sites i and
// i+1 passes no occupied orbital in between, so its amplitude is -t.  The
// ring bond (L-1, 0) passes the other N_s - 1 electrons of that species and
// carries (-1)^(N_s - 1).  The down species never picks up a sign from the up
// orbitals because they are passed twice (once by c, once by c^dag).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <tuple>
#include <mutex>
#include <map>

#include "kernels.cuh"

struct msb_basis {
    int L, n_up, n_dn;
    std::vector<uint32_t> up, dn;
};

namespace msb {

std::vector<uint32_t> sector_states(int L, int n) {
    std::vector<uint32_t> s;
    for (uint32_t v = 0; v < (1u << L); ++v)
        if (__builtin_popcount(v) == n) s.push_back(v);
    return s;  // ascending = rank order
}

std::vector<Bond> lattice_bonds(int L, bool periodic, int lx, bool diag) {
    std::vector<Bond> out;
    if (lx == 0) {
        const int nb = periodic ? L : L - 1;
        for (int i = 0; i < nb; ++i) out.push_back({i, (i + 1) % L, 0});
        return out;
    }
    const int ly = L / lx;
    auto site = [&](int x, int y) { return ((x % lx + lx) % lx) + lx * ((y % ly + ly) % ly); };
    for (int y = 0; y < ly; ++y)
        for (int x = 0; x < lx; ++x) {
            out.push_back({site(x, y), site(x + 1, y), 0});
            out.push_back({site(x, y), site(x, y + 1), 0});
            if (diag) {
                out.push_back({site(x, y), site(x + 1, y + 1), 1});
                out.push_back({site(x, y), site(x - 1, y + 1), 1});
            }
        }
    return out;
}

// ELL hop table of the bonds of class `cls` for one species with n electrons.
// Sign: with all orbitals of one species consecutive in the Jordan-Wigner order,
// a hop between sites a < b passes the occupied orbitals of that species strictly
// between a and b, (-1)^(their number).  (On the ring this is -1 only for the bond
// L-1 -- 0 with an even electron count: (-1)^(N - 1).)
void hop_table_bonds(const std::vector<Bond>& bonds, int cls, int L, int n, const std::vector<uint32_t>& states,
                     std::vector<int32_t>& table, std::vector<uint8_t>& count, int& W, std::vector<uint8_t>* dir) {
    (void)n;
    const int64_t D = int64_t(states.size());
    std::vector<int32_t> rank(size_t(1) << L, -1);
    for (int64_t i = 0; i < D; ++i) rank[states[i]] = int32_t(i);
    std::vector<Bond> bs;
    for (const Bond& b : bonds) if (b.cls == cls) bs.push_back(b);
    const int nb = int(bs.size());
    W = std::max(nb, 1);
    MSB_REQUIRE(W <= 255, "too many bonds for the hop table");
    table.assign(size_t(W) * D, -1);
    count.assign(size_t(D), 0);
    if (dir) dir->assign(size_t(W) * D, 0);
    for (int64_t k = 0; k < D; ++k) {
        const uint32_t s = states[k];
        int c = 0;
        for (const Bond& b : bs) {
            const uint32_t bi = (s >> b.i) & 1u, bj = (s >> b.j) & 1u;
            if (bi == bj) continue;
            const int lo = std::min(b.i, b.j), hi = std::max(b.i, b.j);
            const uint32_t between = ((1u << hi) - 1u) & ~((1u << (lo + 1)) - 1u);
            const bool neg = __builtin_popcount(s & between) & 1;
            const uint32_t tgt = s ^ (1u << b.i) ^ (1u << b.j);
            table[size_t(c) * D + k] = (rank[tgt] << 1) | (neg ? 1 : 0);
            // <s|H|target>: the electron moves from its site in the target to its site in s,
            // i -> j (the bond's direction) when s holds it on j
            if (dir) (*dir)[size_t(c) * D + k] = uint8_t(bj);
            ++c;
        }
        count[k] = uint8_t(c);
    }
}

void hop_table(int L, int n, bool periodic, const std::vector<uint32_t>& states,
               std::vector<int32_t>& table, std::vector<uint8_t>& count, int& W, int lx, std::vector<uint8_t>* dir) {
    hop_table_bonds(lattice_bonds(L, periodic, lx, false), 0, L, n, states, table, count, W, dir);
}

// ---------------------------------------------------------------------------
// Shared-memory placement and hop schedule of a down-spin row for the FP32
// row-tiled apply.
//
// The apply stages row u of V_k in shared memory (lane i stores positions 2i and
// 2i + 1 at their slots; kRowZeroWords zero words follow the row, one on each
// bank pair) and gathers the down-spin hop targets from it: lane l of warp w
// handles positions 2q, 2q + 1 with q = it * threads + 32 w + l, and in round
// k < R_w (R_w = the warp's largest hop count) every lane loads one 8-byte word
// per position, the word the table names for (k, position): one of its hop
// targets, or a zero word in an idle round.  A 32-lane 8-byte access is served
// per half-warp, and distinct words on one bank pair (32 banks of 4 bytes)
// serialise.  The hop table is the same for every row u, so two choices are
// made once per sector, neither of which changes a result beyond the order of
// a sum:
//  1. the slot of each position (a permutation), by simulated annealing over
//     swaps.  A group g = (warp, half-warp, parity) has R_g rounds, so it reads
//     each bank pair at most R_g times without a conflict; the annealer
//     minimises the summed squared excess sum_g sum_b max(0, n_gb - R_g)^2 of
//     the hops n_gb that land on bank pair b, plus, per group, the shortfall of
//     one round with up to two words per bank pair that leaves every bank pair
//     at most R_g - 1 hops (sum_b max(0, n_gb - R_g + 1) must not exceed the
//     lanes), and the same terms for the staging stores (16 positions per set,
//     capacity 1).
//  2. the round of each hop: in each group the hops form a bipartite multigraph,
//     lanes x bank pairs.  y rounds take up to two words per bank pair (each
//     chosen by a feasible flow so that what remains can be finished) and the
//     other R_g - y rounds are a proper edge colouring (Konig), R_g + y
//     wavefronts in all, for the smallest y that works.  An idle round reads
//     the zero word on a bank pair that no hop uses in that round.
// Deterministic (fixed seed).  The reported costs are the mean worst-bank count
// per half-warp gather of the kernel's exact access sets, for the identity slots
// with the table in hop order, and for the chosen slots and rounds.
// ---------------------------------------------------------------------------
namespace {

struct Splitmix {
    uint64_t s;
    uint64_t next() {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double unit() { return double(next() >> 11) * (1.0 / 9007199254740992.0); }
};

// Mean worst-bank distinct-word count over the access sets (warp, half-warp,
// round k < R_w, parity) of the gathers, for table entries tab (k, p) (target
// position << 1 | sign; -1 = the zero word at D) and slots pos (of positions
// 0..D-1 and the zero words D..D+kRowZeroWords-1).
double gather_cost(const std::vector<int32_t>& tab, const std::vector<uint8_t>& count, int64_t D, int threads,
                   const std::vector<int32_t>& pos) {
    const int64_t half = D / 2;
    double sum = 0;
    int64_t nsets = 0;
    int32_t words[16];
    for (int64_t it = 0; it * threads < half; ++it)
        for (int w = 0; w < threads / 32; ++w) {
            const int64_t q0 = it * threads + int64_t(w) * 32;
            if (q0 >= half) continue;
            int R = 0;
            for (int64_t q = q0; q < std::min(q0 + 32, half); ++q)
                R = std::max(R, int(std::max(count[2 * q], count[2 * q + 1])));
            for (int hw = 0; hw < 2; ++hw) {
                const int64_t a = q0 + 16 * hw, b = std::min(a + 16, half);
                if (a >= b) continue;
                for (int k = 0; k < R; ++k)
                    for (int par = 0; par < 2; ++par) {
                        int n = 0;
                        for (int64_t q = a; q < b; ++q) {
                            const int32_t e = tab[size_t(k) * D + 2 * q + par];
                            const int32_t wd = pos[e < 0 ? D : (e >> 1)];
                            bool seen = false;
                            for (int j = 0; j < n; ++j) seen = seen || words[j] == wd;
                            if (!seen) words[n++] = wd;
                        }
                        int c[16] = {0};
                        int m = 0;
                        for (int j = 0; j < n; ++j) m = std::max(m, ++c[words[j] & 15]);
                        sum += m;
                        ++nsets;
                    }
            }
        }
    return nsets ? sum / double(nsets) : 0.0;
}

// Local search over the rounds of one group (a[j * R + r] = slot, -1 idle):
// swaps of two rounds of one lane that do not raise the sum over rounds of the
// worst bank pair's distinct-word count (sideways moves let a conflict join a
// round that already pays for one).  Deterministic.
void polish_rounds(std::vector<int32_t>& a, int nl, int R) {
    if (R <= 1 || nl <= 1) return;
    std::vector<int32_t> wd(size_t(R) * 16 * 16), mu(size_t(R) * 16 * 16);
    std::vector<uint8_t> nw(size_t(R) * 16, 0);
    auto add = [&](int r, int32_t w) {
        if (w < 0) return;
        const int b = w & 15;
        int32_t* Wd = &wd[(size_t(r) * 16 + b) * 16];
        int32_t* M = &mu[(size_t(r) * 16 + b) * 16];
        uint8_t& n = nw[size_t(r) * 16 + b];
        for (int j = 0; j < n; ++j)
            if (Wd[j] == w) { ++M[j]; return; }
        Wd[n] = w;
        M[n] = 1;
        ++n;
    };
    auto del = [&](int r, int32_t w) {
        if (w < 0) return;
        const int b = w & 15;
        int32_t* Wd = &wd[(size_t(r) * 16 + b) * 16];
        int32_t* M = &mu[(size_t(r) * 16 + b) * 16];
        uint8_t& n = nw[size_t(r) * 16 + b];
        for (int j = 0; j < n; ++j)
            if (Wd[j] == w) {
                if (--M[j] == 0) { Wd[j] = Wd[n - 1]; M[j] = M[n - 1]; --n; }
                return;
            }
    };
    auto rcost = [&](int r) {
        int m = 0;
        for (int b = 0; b < 16; ++b) m = std::max(m, int(nw[size_t(r) * 16 + b]));
        return m;
    };
    for (int j = 0; j < nl; ++j)
        for (int r = 0; r < R; ++r) add(r, a[size_t(j) * R + r]);
    Splitmix rng{0x5851F42D4C957F2Dull ^ uint64_t(nl * 131 + R)};
    const int64_t trials = int64_t(1500) * R;
    for (int64_t t = 0; t < trials; ++t) {
        const int j = int(rng.next() % uint64_t(nl));
        const int r1 = int(rng.next() % uint64_t(R)), r2 = int(rng.next() % uint64_t(R));
        int32_t& x = a[size_t(j) * R + r1];
        int32_t& y = a[size_t(j) * R + r2];
        if (r1 == r2 || x == y) continue;
        const int before = rcost(r1) + rcost(r2);
        del(r1, x); add(r1, y);
        del(r2, y); add(r2, x);
        if (rcost(r1) + rcost(r2) <= before) {
            std::swap(x, y);
        } else {
            del(r1, y); add(r1, x);
            del(r2, x); add(r2, y);
        }
    }
}

// Proper edge colouring of a bipartite multigraph (edges e: lane el[e], bank
// pair eb[e]; only edges with col[e] == -1 and !skip[e]) with C colours, every
// vertex of degree <= C, by Kempe-chain flips: for an edge (j, b), colour a free
// at j and c free at b; if neither is free at both ends, the a/c alternating
// path from b is flipped, which frees a at b (the path cannot reach j, which
// misses a).  Colours are written as col[e] = base + colour.
void kempe_colour(const std::vector<int32_t>& el, const std::vector<int32_t>& eb, const std::vector<uint8_t>& skip,
                  std::vector<int32_t>& col, int nl, int C, int base) {
    const int E = int(el.size());
    if (C <= 0) {
        for (int e = 0; e < E; ++e) MSB_REQUIRE(skip[e], "edge colouring without colours");
        return;
    }
    std::vector<int32_t> Lc(size_t(nl) * C, -1), Bc(size_t(16) * C, -1), c(E, -1);
    std::vector<int32_t> path;
    for (int e = 0; e < E; ++e) {
        if (skip[e]) continue;
        const int j = el[e], b = eb[e];
        int ca = 0, cc = 0;
        while (ca < C && Lc[size_t(j) * C + ca] >= 0) ++ca;
        while (cc < C && Bc[size_t(b) * C + cc] >= 0) ++cc;
        MSB_REQUIRE(ca < C && cc < C, "edge colouring ran out of colours");
        int use = -1;
        if (Bc[size_t(b) * C + ca] < 0) use = ca;
        else if (Lc[size_t(j) * C + cc] < 0) use = cc;
        else {
            path.clear();
            int v = b, cur = ca;
            bool at_bank = true;
            for (;;) {
                const int32_t f = at_bank ? Bc[size_t(v) * C + cur] : Lc[size_t(v) * C + cur];
                if (f < 0) break;
                path.push_back(f);
                v = at_bank ? el[f] : eb[f];
                at_bank = !at_bank;
                cur = cur == ca ? cc : ca;
                MSB_REQUIRE(int(path.size()) <= E, "edge colouring path does not end");
            }
            for (int32_t f : path) {
                Lc[size_t(el[f]) * C + c[f]] = -1;
                Bc[size_t(eb[f]) * C + c[f]] = -1;
            }
            for (int32_t f : path) {
                c[f] = c[f] == ca ? cc : ca;
                Lc[size_t(el[f]) * C + c[f]] = f;
                Bc[size_t(eb[f]) * C + c[f]] = f;
            }
            MSB_REQUIRE(Bc[size_t(b) * C + ca] < 0 && Lc[size_t(j) * C + ca] < 0, "edge colouring flip failed");
            use = ca;
        }
        c[e] = use;
        Lc[size_t(j) * C + use] = e;
        Bc[size_t(b) * C + use] = e;
    }
    for (int e = 0; e < E; ++e)
        if (!skip[e]) col[e] = base + c[e];
}

// One round peeled off a group (edges with live[e]): one hop per lane of
// remaining degree `left` (at most one for the others), and per bank pair b
// between max(0, deg_b - keep) and `cap` hops, so that afterwards every lane has
// degree <= left - 1 and every bank pair <= keep.  A feasible flow with lower
// bounds (source -> lanes -> bank pairs -> sink, circulation edge sink ->
// source, the bounds moved to a super source and sink), augmenting paths by
// depth-first search.  Returns false if no such round exists.
bool peel_round(const std::vector<int32_t>& el, const std::vector<int32_t>& eb, const std::vector<uint8_t>& live,
                int nl, int left, int keep, int cap_b, std::vector<int32_t>& pick) {
    const int E = int(el.size());
    int degl[16] = {0}, degb[16] = {0}, mult[16][16] = {{0}};
    for (int e = 0; e < E; ++e)
        if (live[e]) { ++degl[el[e]]; ++degb[eb[e]]; ++mult[el[e]][eb[e]]; }
    const int S = 0, L0 = 1, B0 = 1 + nl, T = B0 + 16, SS = T + 1, TT = T + 2, N = T + 3;
    std::vector<int> cap(size_t(N) * N, 0), exc(N, 0);
    auto edge = [&](int u, int v, int lo, int hi) {
        cap[size_t(u) * N + v] += hi - lo;
        exc[v] += lo;
        exc[u] -= lo;
    };
    for (int j = 0; j < nl; ++j) {
        if (degl[j] > left) return false;
        edge(S, L0 + j, degl[j] == left ? 1 : 0, degl[j] > 0 ? 1 : 0);
    }
    for (int j = 0; j < nl; ++j)
        for (int b = 0; b < 16; ++b)
            if (mult[j][b]) edge(L0 + j, B0 + b, 0, mult[j][b]);
    for (int b = 0; b < 16; ++b) {
        const int lo = std::max(0, degb[b] - keep), hi = std::min(cap_b, degb[b]);
        if (lo > hi) return false;
        edge(B0 + b, T, lo, hi);
    }
    edge(T, S, 0, 1 << 20);
    int need = 0;
    for (int v = 0; v < N; ++v) {
        if (exc[v] > 0) { cap[size_t(SS) * N + v] += exc[v]; need += exc[v]; }
        else if (exc[v] < 0) cap[size_t(v) * N + TT] += -exc[v];
    }
    std::vector<int> seen(N), stack, parent(N);
    int flow = 0;
    for (;;) {
        std::fill(seen.begin(), seen.end(), 0);
        stack.assign(1, SS);
        seen[SS] = 1;
        while (!stack.empty() && !seen[TT]) {
            const int u = stack.back();
            stack.pop_back();
            for (int v = 0; v < N; ++v)
                if (!seen[v] && cap[size_t(u) * N + v] > 0) { seen[v] = 1; parent[v] = u; stack.push_back(v); }
        }
        if (!seen[TT]) break;
        for (int v = TT; v != SS; v = parent[v]) {
            --cap[size_t(parent[v]) * N + v];
            ++cap[size_t(v) * N + parent[v]];
        }
        ++flow;
    }
    if (flow < need) return false;
    // lane -> bank pair units used: the original capacity less the residual
    pick.assign(E, 0);
    for (int j = 0; j < nl; ++j)
        for (int b = 0; b < 16; ++b) {
            int used = mult[j][b] - cap[size_t(L0 + j) * N + B0 + b];
            for (int e = 0; e < E && used > 0; ++e)
                if (live[e] && el[e] == j && eb[e] == b && !pick[e]) { pick[e] = 1; --used; }
        }
    return true;
}

// The rounds of one group (nl <= 16 lanes, R rounds).  In: a[j * R + k] = the
// slot of lane j's k-th hop, or -1 past its hop count.  Out: a[j * R + r] = the
// slot lane j reads in round r, zero words (slots zero0 + b) in idle rounds.
// y rounds take up to two words per bank pair (peel_round, one at a time) and
// the other R - y rounds are a proper colouring (kempe_colour): R + y
// wavefronts, for the smallest y that works (at least the largest excess x of
// a bank pair's hops over R: no order does better than R + x).  A local search
// then lets conflicts share rounds and lanes reading one word share a round.
void schedule_group(std::vector<int32_t>& a, int nl, int R, int32_t zero0) {
    if (R <= 0 || nl <= 0) return;
    std::vector<int32_t> el, eb, ew;                   // lane, bank pair, slot of each hop
    std::vector<int32_t> byb[16];
    for (int j = 0; j < nl; ++j)
        for (int r = 0; r < R; ++r) {
            const int32_t w = a[size_t(j) * R + r];
            if (w < 0) continue;
            byb[w & 15].push_back(int32_t(el.size()));
            el.push_back(j);
            eb.push_back(w & 15);
            ew.push_back(w);
        }
    const int E = int(el.size());
    int x = 0;
    for (int b = 0; b < 16; ++b) x = std::max(x, int(byb[b].size()) - R);
    std::vector<int32_t> col(E, -1), pick;
    std::vector<uint8_t> held(E, 0), live(E);
    // y rounds that take up to two words per bank pair, then a proper colouring
    // of the rest with R - y colours; the smallest y that works
    bool done = false;
    for (int y = x; y < R && !done; ++y) {
        std::fill(live.begin(), live.end(), 1);
        std::fill(col.begin(), col.end(), -1);
        bool ok = true;
        for (int i = 0; i < y && ok; ++i) {
            // after this round: lanes <= R - i - 1, bank pairs <= (R - y) + 2 (y - i - 1)
            ok = peel_round(el, eb, live, nl, R - i, (R - y) + 2 * (y - i - 1), 2, pick);
            if (ok)
                for (int e = 0; e < E; ++e)
                    if (pick[e]) { col[e] = i; live[e] = 0; }
        }
        if (!ok) continue;
        std::vector<uint8_t> skip(E);
        for (int e = 0; e < E; ++e) skip[e] = !live[e];
        kempe_colour(el, eb, skip, col, nl, R - y, y);
        done = true;
    }
    if (!done) {
        // fall back: an R-colouring of the hops up to R per bank pair, the rest
        // placed where they cost least
        std::fill(col.begin(), col.end(), -1);
        for (int b = 0; b < 16; ++b) {
            int excess = int(byb[b].size()) - R;
            for (int i = int(byb[b].size()) - 1; i >= 0 && excess > 0; --i) { held[byb[b][i]] = 1; --excess; }
        }
        kempe_colour(el, eb, held, col, nl, R, 0);
    }
    for (int j = 0; j < nl; ++j)
        for (int r = 0; r < R; ++r) a[size_t(j) * R + r] = -1;
    std::vector<std::vector<int32_t>> words(size_t(R) * 16);
    std::vector<int> rmax(R, 0);
    auto put = [&](int j, int r, int32_t w) {
        MSB_REQUIRE(a[size_t(j) * R + r] < 0, "two hops of a lane in one round");
        a[size_t(j) * R + r] = w;
        auto& v = words[size_t(r) * 16 + (w & 15)];
        if (std::find(v.begin(), v.end(), w) == v.end()) v.push_back(w);
        rmax[r] = std::max(rmax[r], int(v.size()));
    };
    for (int e = 0; e < E; ++e)
        if (!held[e]) put(el[e], col[e], ew[e]);
    for (int e = 0; e < E; ++e) {
        if (!held[e]) continue;
        const int j = el[e], b = eb[e];
        int best = -1, bcost = 0, bn = 0;
        for (int r = 0; r < R; ++r) {
            if (a[size_t(j) * R + r] >= 0) continue;
            const auto& v = words[size_t(r) * 16 + b];
            const bool has = std::find(v.begin(), v.end(), ew[e]) != v.end();
            const int n = has ? int(v.size()) : int(v.size()) + 1;
            const int cost = std::max(0, n - std::max(rmax[r], 1));
            if (best < 0 || cost < bcost || (cost == bcost && n < bn)) { best = r; bcost = cost; bn = n; }
        }
        MSB_REQUIRE(best >= 0, "no free round for a hop");
        put(j, best, ew[e]);
    }
    polish_rounds(a, nl, R);
    // idle rounds: the zero word on a bank pair no hop of the round uses (one
    // exists: an idle lane leaves at most 15 words in the round)
    for (auto& v : words) v.clear();
    for (int j = 0; j < nl; ++j)
        for (int r = 0; r < R; ++r) {
            const int32_t w = a[size_t(j) * R + r];
            if (w < 0) continue;
            auto& v = words[size_t(r) * 16 + (w & 15)];
            if (std::find(v.begin(), v.end(), w) == v.end()) v.push_back(w);
        }
    for (int r = 0; r < R; ++r) {
        int fb = -1;
        for (int b = 0; b < 16 && fb < 0; ++b)
            if (words[size_t(r) * 16 + b].empty()) fb = b;
        for (int j = 0; j < nl; ++j) {
            if (a[size_t(j) * R + r] >= 0) continue;
            MSB_REQUIRE(fb >= 0, "no free bank pair for an idle round");
            a[size_t(j) * R + r] = zero0 + ((fb - zero0) & 15);
        }
    }
}

}  // namespace

RowLayout row_layout(const std::vector<int32_t>& table, const std::vector<uint8_t>& count, int64_t D, int W,
                     int threads) {
    MSB_REQUIRE(D >= 2 && D % 2 == 0 && D + kRowZeroWords < 32768, "row layout needs an even D < 32752");
    MSB_REQUIRE(threads >= 32 && threads % 32 == 0, "threads must be a multiple of 32");
    const int64_t half = D / 2;
    // sets: the gather groups (hops with their multiplicities, capacity R_g) and
    // the staging stores (16 positions of one parity, capacity 1)
    std::vector<int32_t> mem, mul;
    std::vector<int64_t> beg{0};
    std::vector<int32_t> cap;
    struct Group { int64_t a, b; int par, R; };
    std::vector<Group> groups;
    std::vector<int32_t> tmp;
    for (int64_t it = 0; it * threads < half; ++it)
        for (int w = 0; w < threads / 32; ++w) {
            const int64_t q0 = it * threads + int64_t(w) * 32;
            if (q0 >= half) continue;
            int R = 0;
            for (int64_t q = q0; q < std::min(q0 + 32, half); ++q)
                R = std::max(R, int(std::max(count[2 * q], count[2 * q + 1])));
            for (int hw = 0; hw < 2; ++hw) {
                const int64_t a = q0 + 16 * hw, b = std::min(a + 16, half);
                if (a >= b) continue;
                for (int par = 0; par < 2; ++par) {
                    groups.push_back({a, b, par, R});
                    tmp.clear();
                    for (int64_t q = a; q < b; ++q)
                        for (int k = 0; k < count[2 * q + par]; ++k) tmp.push_back(table[size_t(k) * D + 2 * q + par] >> 1);
                    std::sort(tmp.begin(), tmp.end());
                    for (size_t i = 0; i < tmp.size();) {
                        size_t j = i;
                        while (j < tmp.size() && tmp[j] == tmp[i]) ++j;
                        mem.push_back(tmp[i]);
                        mul.push_back(int32_t(j - i));
                        i = j;
                    }
                    beg.push_back(int64_t(mem.size()));
                    cap.push_back(R);
                }
            }
        }
    for (int64_t i0 = 0; i0 < half; i0 += 16)
        for (int par = 0; par < 2; ++par) {
            for (int64_t i = i0; i < std::min(i0 + 16, half); ++i) {
                mem.push_back(int32_t(2 * i + par));
                mul.push_back(1);
            }
            beg.push_back(int64_t(mem.size()));
            cap.push_back(1);
        }
    const int64_t nsets = int64_t(beg.size()) - 1;
    // lanes of each set: a round with two words per bank pair takes one hop per lane
    std::vector<int32_t> lanes(static_cast<size_t>(nsets));
    for (int64_t si = 0; si < nsets; ++si)
        lanes[si] = si < int64_t(groups.size()) ? int32_t(groups[si].b - groups[si].a) : int32_t(beg[si + 1] - beg[si]);
    std::vector<std::vector<std::pair<int32_t, int32_t>>> sets_of(static_cast<size_t>(D));
    for (int64_t si = 0; si < nsets; ++si)
        for (int64_t j = beg[si]; j < beg[si + 1]; ++j) sets_of[mem[j]].push_back({int32_t(si), mul[j]});
    std::vector<int32_t> pos(size_t(D) + kRowZeroWords);
    // start: position 2i + par with i = 16 m + l at slot 32 m + 16 par + l, so that
    // every full staging store set covers the 16 bank pairs once (the last,
    // partial block keeps slot = position); swaps stay inside a store set
    for (int64_t e = 0; e < D + kRowZeroWords; ++e) pos[e] = int32_t(e);
    const int64_t full = half / 16 * 16;
    for (int64_t i = 0; i < full; ++i)
        for (int par = 0; par < 2; ++par) pos[2 * i + par] = int32_t(32 * (i / 16) + 16 * par + (i % 16));
    std::vector<int16_t> cnt(size_t(nsets) * 16, 0);
    for (int64_t si = 0; si < nsets; ++si)
        for (int64_t j = beg[si]; j < beg[si + 1]; ++j) cnt[size_t(si) * 16 + (pos[mem[j]] & 15)] += int16_t(mul[j]);
    // cost of a set: the squared excess of each bank pair over the capacity R,
    // plus the shortfall of a round with up to two words per bank pair after
    // which every bank pair holds at most R - 1: sum_b max(0, n_b - R + 1) hops
    // must fit one per lane
    auto pen = [](int c, int R) { const int x = c > R ? c - R : 0; return x * x; };
    auto need = [](int c, int R) { return c > R - 1 ? c - R + 1 : 0; };
    std::vector<int32_t> needs(size_t(nsets), 0);
    for (int64_t si = 0; si < nsets; ++si)
        for (int b = 0; b < 16; ++b) needs[si] += need(cnt[size_t(si) * 16 + b], cap[si]);
    std::vector<int64_t> stamp(size_t(nsets), -1);
    std::vector<int32_t> mx(size_t(nsets), 0);
    Splitmix rng{0x9E3779B97F4A7C15ull};
    struct Touch { int32_t si, d, dn; };                     // set, change on x's bank pair, change of needs
    std::vector<Touch> touched;
    // simulated annealing over swaps: a worsening swap is taken with probability
    // exp(-delta / T), the temperature falling to zero over the trials
    const int64_t trials = 1000 * D;
    const double T0 = 1.0;
    for (int64_t t = 0; t < trials; ++t) {
        const int32_t x = int32_t(rng.next() % uint64_t(D));
        const int64_t i0 = (x >> 1) / 16 * 16, n0 = std::min<int64_t>(16, half - i0);
        const int32_t y = int32_t(2 * (i0 + int64_t(rng.next() % uint64_t(n0))) + (x & 1));
        const int bx = pos[x] & 15, by = pos[y] & 15;
        if (bx == by) continue;
        // after the swap x sits on by and y on bx: a set holding x m_x times and y
        // m_y times changes its count on bx by d = m_y - m_x and on by by -d
        for (const auto& sm : sets_of[x]) { stamp[sm.first] = 2 * t; mx[sm.first] = sm.second; }
        long delta = 0;
        touched.clear();
        auto consider = [&](int32_t si, int d) {
            if (d == 0) return;
            const int16_t* c = &cnt[size_t(si) * 16];
            const int R = cap[si];
            delta += pen(c[bx] + d, R) - pen(c[bx], R) + pen(c[by] - d, R) - pen(c[by], R);
            const int dn = need(c[bx] + d, R) - need(c[bx], R) + need(c[by] - d, R) - need(c[by], R);
            delta += std::max(0, needs[si] + dn - lanes[si]) - std::max(0, needs[si] - lanes[si]);
            touched.push_back({si, d, dn});
        };
        for (const auto& sm : sets_of[y]) {
            if (stamp[sm.first] == 2 * t) { stamp[sm.first] = 2 * t + 1; consider(sm.first, sm.second - mx[sm.first]); }
            else consider(sm.first, sm.second);
        }
        for (const auto& sm : sets_of[x])
            if (stamp[sm.first] == 2 * t) consider(sm.first, -sm.second);
        bool take = delta <= 0;
        if (!take) {
            const double f = 1.0 - double(t) / double(trials);
            const double T = T0 * f * f;
            take = T > 0 && rng.unit() < std::exp(-double(delta) / T);
        }
        if (!take) continue;
        for (const Touch& td : touched) {
            int16_t* c = &cnt[size_t(td.si) * 16];
            c[bx] += int16_t(td.d);
            c[by] -= int16_t(td.d);
            needs[td.si] += td.dn;
        }
        std::swap(pos[x], pos[y]);
    }
    RowLayout out;
    out.perm.resize(size_t(D));
    std::vector<uint8_t> seen(size_t(D), 0);
    for (int64_t e = 0; e < D; ++e) {
        MSB_REQUIRE(pos[e] >= 0 && pos[e] < D && !seen[pos[e]], "row layout is not a permutation");
        seen[pos[e]] = 1;
        out.perm[e] = uint16_t(pos[e]);
    }
    // the rounds of every group, on the chosen slots; table entries in position
    // space (a zero word's position is its slot)
    std::vector<int32_t> inv(size_t(D) + kRowZeroWords);
    for (int64_t e = 0; e < D + kRowZeroWords; ++e) inv[pos[e]] = int32_t(e);
    out.width = W;
    out.table.assign(size_t(W) * D, int32_t(D) << 1);
    std::vector<int32_t> a;
    for (const Group& g : groups) {
        const int nl = int(g.b - g.a), R = g.R;
        MSB_REQUIRE(R <= W, "hop count above the table width");
        a.assign(size_t(nl) * R, -1);
        for (int j = 0; j < nl; ++j) {
            const int64_t p = 2 * (g.a + j) + g.par;
            for (int k = 0; k < count[p]; ++k) a[size_t(j) * R + k] = pos[table[size_t(k) * D + p] >> 1];
        }
        schedule_group(a, nl, R, int32_t(D));
        for (int j = 0; j < nl; ++j) {
            const int64_t p = 2 * (g.a + j) + g.par;
            std::vector<uint8_t> used(count[p], 0);
            for (int r = 0; r < R; ++r) {
                const int32_t t = inv[a[size_t(j) * R + r]];
                int32_t e = t << 1;                              // a zero word
                if (t < D) {
                    e = -1;
                    for (int k = 0; k < count[p] && e < 0; ++k) {
                        const int32_t c = table[size_t(k) * D + p];
                        if (!used[k] && (c >> 1) == t) { used[k] = 1; e = c; }
                    }
                    MSB_REQUIRE(e >= 0, "hop schedule names a word that is not a hop");
                }
                out.table[size_t(r) * D + p] = e;
            }
            for (int k = 0; k < count[p]; ++k) MSB_REQUIRE(used[k], "hop schedule lost a hop");
        }
    }
    std::vector<int32_t> ident(size_t(D) + kRowZeroWords);
    for (int64_t e = 0; e < D + kRowZeroWords; ++e) ident[e] = int32_t(e);
    out.cost_plain = gather_cost(table, count, D, threads, ident);
    out.cost_layout = gather_cost(out.table, count, D, threads, pos);
    return out;
}

// ---------------------------------------------------------------------------
// Row order of the continued fraction.  The second step only needs the
// Lanczos coefficients, so its vectors may hold each row's down-spin states in
// any fixed order.  The row-tiled apply runs its down-spin loop to the largest
// hop count of the 32 (FP64) or 64 (FP32) elements of a warp; in rank order a
// warp's largest count is ~40% above the mean (L = 14: 10.5 vs 7.5).  Position
// p of a row therefore holds down state order[p], with the states sorted by
// hop count (descending, ties in rank order): a warp's elements then have
// (nearly) equal counts.
// ---------------------------------------------------------------------------
std::vector<uint16_t> row_order(const std::vector<uint8_t>& count) {
    const int64_t D = int64_t(count.size());
    MSB_REQUIRE(D >= 1 && D < 65536, "row order needs fewer than 65536 states");
    std::vector<uint16_t> ord(static_cast<size_t>(D));
    for (int64_t i = 0; i < D; ++i) ord[i] = uint16_t(i);
    std::stable_sort(ord.begin(), ord.end(), [&](uint16_t a, uint16_t b) { return count[a] > count[b]; });
    return ord;
}

// The rank-space hop table rewritten to positions: entry (p, slot k) targets
// position inv[t] for the k-th hop t of state order[p] (sign bit kept).
void table_in_row_order(const std::vector<int32_t>& table, const std::vector<uint8_t>& count, int64_t D, int W,
                        const std::vector<uint16_t>& ord, std::vector<int32_t>& tpos, std::vector<uint8_t>& cpos) {
    std::vector<int32_t> inv(static_cast<size_t>(D));
    for (int64_t p = 0; p < D; ++p) inv[ord[p]] = int32_t(p);
    tpos.assign(size_t(W) * D, -1);
    cpos.assign(size_t(D), 0);
    for (int64_t p = 0; p < D; ++p) {
        const int64_t d = ord[p];
        cpos[p] = count[d];
        for (int k = 0; k < count[d]; ++k) {
            const int32_t e = table[size_t(k) * D + d];
            tpos[size_t(k) * D + p] = (inv[e >> 1] << 1) | (e & 1);
        }
    }
}

const std::vector<uint16_t>& cached_row_order(int L, int n, bool periodic, int lx) {
    static std::mutex mu;
    static std::map<std::tuple<int, int, bool, int>, std::vector<uint16_t>> cache;
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_tuple(L, n, periodic, lx);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    const auto states = sector_states(L, n);
    std::vector<int32_t> table;
    std::vector<uint8_t> count;
    int W = 0;
    hop_table(L, n, periodic, states, table, count, W, lx);
    return cache.emplace(key, row_order(count)).first->second;
}

// Bank-aware placement of the row in its continued-fraction order (the kernel
// gathers by position).
const RowLayout& cached_row_layout(int L, int n, bool periodic, int threads, int lx) {
    static std::mutex mu;
    static std::map<std::tuple<int, int, bool, int, int>, RowLayout> cache;
    const auto& ord = cached_row_order(L, n, periodic, lx);
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_tuple(L, n, periodic, threads, lx);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    const auto states = sector_states(L, n);
    std::vector<int32_t> table, tpos;
    std::vector<uint8_t> count, cpos;
    int W = 0;
    hop_table(L, n, periodic, states, table, count, W, lx);
    table_in_row_order(table, count, int64_t(states.size()), W, ord, tpos, cpos);
    return cache.emplace(key, row_layout(tpos, cpos, int64_t(states.size()), W, threads)).first->second;
}

void validate_model(const msb_model& m) {
    MSB_REQUIRE(m.L >= 2 && m.L <= 16, "model.L must be in 2..16");
    MSB_REQUIRE(!(m.periodic && m.L < 3), "a periodic chain needs L >= 3");
    MSB_REQUIRE(m.n_up >= 0 && m.n_up <= m.L && m.n_dn >= 0 && m.n_dn <= m.L,
                "electron counts must be in 0..L");
    MSB_REQUIRE(m.core_site >= 0 && m.core_site < m.L, "core_site must be in 0..L-1");
    MSB_REQUIRE((m.o2_spin == 0 || m.o2_spin == 1) && (m.o1_spin == 0 || m.o1_spin == 1),
                "o2_spin and o1_spin must be 0 (up) or 1 (down)");
    MSB_REQUIRE(m.lx == 0 || (m.lx >= 3 && m.L % m.lx == 0 && m.L / m.lx >= 3),
                "a 2D cluster needs lx >= 3 dividing L with L / lx >= 3");
    MSB_REQUIRE(std::isfinite(m.tp) && (m.tp == 0.0 || m.lx > 0), "tp needs a 2D cluster (lx > 0)");
    MSB_REQUIRE(std::isfinite(m.flux) && (m.flux == 0.0 || m.lx == 0), "a flux needs a chain (lx = 0)");
}

}  // namespace msb

// ----------------------------------------------------------------------------
// C ABI: basis
// ----------------------------------------------------------------------------

extern "C" msb_status msb_basis_create(int L, int n_up, int n_dn, msb_basis** out) {
    return msb::guard("msb_basis_create", [&] {
        MSB_REQUIRE(out != nullptr, "out is NULL");
        MSB_REQUIRE(L >= 1 && L <= 16, "L must be in 1..16");
        MSB_REQUIRE(n_up >= 0 && n_up <= L && n_dn >= 0 && n_dn <= L, "electron counts must be in 0..L");
        auto* b = new msb_basis{L, n_up, n_dn, msb::sector_states(L, n_up), msb::sector_states(L, n_dn)};
        *out = b;
    });
}

extern "C" msb_status msb_basis_dims(const msb_basis* b, int64_t* D_up, int64_t* D_dn, int64_t* dim) {
    return msb::guard("msb_basis_dims", [&] {
        MSB_REQUIRE(b != nullptr, "basis is NULL");
        if (D_up) *D_up = int64_t(b->up.size());
        if (D_dn) *D_dn = int64_t(b->dn.size());
        if (dim) *dim = int64_t(b->up.size()) * int64_t(b->dn.size());
    });
}

extern "C" msb_status msb_basis_states(const msb_basis* b, int species, uint32_t* out) {
    return msb::guard("msb_basis_states", [&] {
        MSB_REQUIRE(b != nullptr && out != nullptr, "NULL argument");
        MSB_REQUIRE(species == 0 || species == 1, "species must be 0 (up) or 1 (down)");
        const auto& v = species == 0 ? b->up : b->dn;
        std::memcpy(out, v.data(), v.size() * sizeof(uint32_t));
    });
}

extern "C" void msb_basis_destroy(msb_basis* b) { delete b; }

extern "C" msb_status msb_basis_row_order(const msb_basis* b, int periodic, uint16_t* order) {
    return msb::guard("msb_basis_row_order", [&] {
        MSB_REQUIRE(b != nullptr && order != nullptr, "NULL argument");
        MSB_REQUIRE(b->dn.size() < 32768, "the row order needs D_dn below 32768");
        MSB_REQUIRE(!(periodic && b->L < 3), "a periodic chain needs L >= 3");
        const auto& ord = msb::cached_row_order(b->L, b->n_dn, periodic != 0);
        std::memcpy(order, ord.data(), ord.size() * sizeof(uint16_t));
    });
}

extern "C" msb_status msb_basis_row_layout(const msb_basis* b, int periodic, uint16_t* slot, int* width,
                                           uint16_t* hops, double* cost_plain, double* cost_layout) {
    return msb::guard("msb_basis_row_layout", [&] {
        MSB_REQUIRE(b != nullptr, "basis is NULL");
        const int64_t D = int64_t(b->dn.size());
        MSB_REQUIRE(D >= 2 && D % 2 == 0 && D + msb::kRowZeroWords < 32768, "the row layout needs an even D_dn below 32752");
        MSB_REQUIRE(!(periodic && b->L < 3), "a periodic chain needs L >= 3");
        const auto& lay = msb::cached_row_layout(b->L, b->n_dn, periodic != 0, msb::kApplyThreads);
        if (slot) std::memcpy(slot, lay.perm.data(), lay.perm.size() * sizeof(uint16_t));
        if (width) *width = lay.width;
        if (hops)
            for (size_t i = 0; i < lay.table.size(); ++i)
                hops[i] = uint16_t(lay.table[i]);
        if (cost_plain) *cost_plain = lay.cost_plain;
        if (cost_layout) *cost_layout = lay.cost_layout;
    });
}
