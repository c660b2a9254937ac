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
// Shared-memory placement of a down-spin row for the FP32 row-tiled apply.
//
// The apply stages row u of V_k in shared memory and gathers the down-spin hop
// targets from it: lane l of warp w handles elements 2q, 2q+1 with
// q = it * threads + 32 w + l, and at hop slot k every lane loads one 8-byte word
// per element (the zero slot at index D once the element's own hops are done;
// the trip count is the warp's largest hop count).  A 32-lane 8-byte load is
// served per half-warp, and two different words on one bank pair (32 banks of
// 4 bytes) serialise.  The hop table is the same for every row u, so the slot of
// each element can be chosen once per sector: a hill climb over swaps of two
// elements on different bank pairs lowers the summed worst-bank count of all
// the access sets.  Deterministic (fixed seed).
// ---------------------------------------------------------------------------
RowLayout row_layout(const std::vector<int32_t>& table, const std::vector<uint8_t>& count, int64_t D, int W,
                     int threads) {
    MSB_REQUIRE(D >= 2 && D % 2 == 0 && D < 32768, "row layout needs an even D < 32768");
    MSB_REQUIRE(threads >= 32 && threads % 32 == 0, "threads must be a multiple of 32");
    const int64_t half = D / 2;
    const int32_t ZERO = int32_t(D);
    // access sets: one per (half-warp, slot, parity), unique members
    std::vector<int32_t> mem;              // concatenated members
    std::vector<int64_t> beg{0};
    std::vector<int32_t> tmp;
    const int64_t iters = (half + threads - 1) / threads;
    for (int64_t it = 0; it < iters; ++it)
        for (int w = 0; w < threads / 32; ++w) {
            const int64_t q0 = it * threads + int64_t(w) * 32;
            if (q0 >= half) continue;
            int ndw = 0;
            for (int l = 0; l < 32 && q0 + l < half; ++l)
                ndw = std::max(ndw, int(std::max(count[2 * (q0 + l)], count[2 * (q0 + l) + 1])));
            for (int hw = 0; hw < 2; ++hw)
                for (int k = 0; k < ndw; ++k)
                    for (int par = 0; par < 2; ++par) {
                        tmp.clear();
                        for (int l = 0; l < 16; ++l) {
                            const int64_t q = q0 + hw * 16 + l;
                            if (q >= half) break;
                            const int64_t d = 2 * q + par;
                            tmp.push_back(k < count[d] ? (table[size_t(k) * D + d] >> 1) : ZERO);
                        }
                        if (tmp.empty()) continue;
                        std::sort(tmp.begin(), tmp.end());
                        tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
                        mem.insert(mem.end(), tmp.begin(), tmp.end());
                        beg.push_back(int64_t(mem.size()));
                    }
        }
    (void)W;
    const int64_t nsets = int64_t(beg.size()) - 1;
    std::vector<std::vector<int32_t>> sets_of(static_cast<size_t>(D));
    for (int64_t si = 0; si < nsets; ++si)
        for (int64_t j = beg[si]; j < beg[si + 1]; ++j)
            if (mem[j] != ZERO) sets_of[mem[j]].push_back(int32_t(si));
    std::vector<int32_t> pos(size_t(D) + 1);
    for (int64_t e = 0; e <= D; ++e) pos[e] = int32_t(e);
    std::vector<uint8_t> cnt(size_t(nsets) * 16, 0);
    std::vector<uint8_t> cur(size_t(nsets), 0);
    auto setmax = [&](int64_t si) {
        uint8_t m = 0;
        for (int b = 0; b < 16; ++b) m = std::max(m, cnt[size_t(si) * 16 + b]);
        return m;
    };
    double plain = 0;
    for (int64_t si = 0; si < nsets; ++si) {
        for (int64_t j = beg[si]; j < beg[si + 1]; ++j) ++cnt[size_t(si) * 16 + (pos[mem[j]] & 15)];
        cur[si] = setmax(si);
        plain += cur[si];
    }
    double total = plain;
    std::vector<int64_t> stamp(size_t(nsets), -1);
    uint64_t rs = 0x9E3779B97F4A7C15ull;
    auto rnd = [&]() {                         // splitmix64
        uint64_t z = (rs += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    std::vector<int32_t> touched;
    // simulated annealing over swaps: a worsening swap is taken with probability
    // exp(-delta / T), the temperature falling to zero over the trials
    const int64_t trials = 1000 * D;
    const double T0 = 0.6;
    for (int64_t t = 0; t < trials; ++t) {
        const int32_t x = int32_t(rnd() % uint64_t(D)), y = int32_t(rnd() % uint64_t(D));
        const int bx = pos[x] & 15, by = pos[y] & 15;
        if (bx == by) continue;
        for (int32_t si : sets_of[x]) stamp[si] = 2 * t;          // sets of x
        touched.clear();
        long delta = 0;
        for (int32_t si : sets_of[y]) {
            if (stamp[si] == 2 * t) { stamp[si] = 2 * t + 1; continue; }   // holds both: unchanged
            uint8_t* c = &cnt[size_t(si) * 16];
            --c[by]; ++c[bx];
            touched.push_back(si);
        }
        for (int32_t si : sets_of[x]) {
            if (stamp[si] != 2 * t) continue;
            uint8_t* c = &cnt[size_t(si) * 16];
            --c[bx]; ++c[by];
            touched.push_back(si);
        }
        for (int32_t si : touched) delta += long(setmax(si)) - long(cur[si]);
        bool take = delta <= 0;
        if (!take) {
            const double f = 1.0 - double(t) / double(trials);
            const double T = T0 * f * f;
            const double u = double(rnd() >> 11) * (1.0 / 9007199254740992.0);
            take = T > 0 && u < std::exp(-double(delta) / T);
        }
        if (take) {
            for (int32_t si : touched) cur[si] = setmax(si);
            std::swap(pos[x], pos[y]);
            total += double(delta);
        } else {                                                // undo
            for (int32_t si : sets_of[y]) {
                if (stamp[si] == 2 * t + 1) continue;
                uint8_t* c = &cnt[size_t(si) * 16];
                ++c[by]; --c[bx];
            }
            for (int32_t si : sets_of[x]) {
                if (stamp[si] != 2 * t) continue;
                uint8_t* c = &cnt[size_t(si) * 16];
                ++c[bx]; --c[by];
            }
        }
    }
    RowLayout out;
    out.perm.resize(size_t(D));
    std::vector<uint8_t> seen(size_t(D), 0);
    for (int64_t e = 0; e < D; ++e) {
        MSB_REQUIRE(pos[e] >= 0 && pos[e] < D && !seen[pos[e]], "row layout is not a permutation");
        seen[pos[e]] = 1;
        out.perm[e] = uint16_t(pos[e]);
    }
    out.cost_plain = nsets ? plain / double(nsets) : 0.0;
    out.cost_layout = nsets ? total / double(nsets) : 0.0;
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

extern "C" msb_status msb_basis_row_layout(const msb_basis* b, int periodic, uint16_t* slot, double* cost_plain,
                                           double* cost_layout) {
    return msb::guard("msb_basis_row_layout", [&] {
        MSB_REQUIRE(b != nullptr, "basis is NULL");
        const int64_t D = int64_t(b->dn.size());
        MSB_REQUIRE(D >= 2 && D % 2 == 0 && D < 32768, "the row layout needs an even D_dn below 32768");
        MSB_REQUIRE(!(periodic && b->L < 3), "a periodic chain needs L >= 3");
        const auto& lay = msb::cached_row_layout(b->L, b->n_dn, periodic != 0, msb::kApplyThreads);
        if (slot) std::memcpy(slot, lay.perm.data(), lay.perm.size() * sizeof(uint16_t));
        if (cost_plain) *cost_plain = lay.cost_plain;
        if (cost_layout) *cost_layout = lay.cost_layout;
    });
}
