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
#include <cstring>

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

void hop_table(int L, int n, bool periodic, const std::vector<uint32_t>& states,
               std::vector<int32_t>& table, std::vector<uint8_t>& count, int& W) {
    const int64_t D = int64_t(states.size());
    std::vector<int32_t> rank(size_t(1) << L, -1);
    for (int64_t i = 0; i < D; ++i) rank[states[i]] = int32_t(i);
    const int nb = periodic ? L : L - 1;
    W = std::max(nb, 1);
    table.assign(size_t(W) * D, -1);
    count.assign(size_t(D), 0);
    const bool ring_neg = periodic && ((n - 1) & 1);
    for (int64_t k = 0; k < D; ++k) {
        const uint32_t s = states[k];
        int c = 0;
        for (int i = 0; i < nb; ++i) {
            const int j = (i + 1) % L;
            const uint32_t bi = (s >> i) & 1u, bj = (s >> j) & 1u;
            if (bi == bj) continue;
            const uint32_t tgt = s ^ (1u << i) ^ (1u << j);
            const bool neg = (j == 0) && ring_neg;
            table[size_t(c) * D + k] = (rank[tgt] << 1) | (neg ? 1 : 0);
            ++c;
        }
        count[k] = uint8_t(c);
    }
}

void validate_model(const msb_model& m) {
    MSB_REQUIRE(m.L >= 2 && m.L <= 16, "model.L must be in 2..16");
    MSB_REQUIRE(!(m.periodic && m.L < 3), "a periodic chain needs L >= 3");
    MSB_REQUIRE(m.n_up >= 0 && m.n_up <= m.L && m.n_dn >= 0 && m.n_dn <= m.L,
                "electron counts must be in 0..L");
    MSB_REQUIRE(m.core_site >= 0 && m.core_site < m.L, "core_site must be in 0..L-1");
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
