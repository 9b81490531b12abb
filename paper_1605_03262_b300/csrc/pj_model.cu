// Host side: reader of the binary kinetic-model format and builder of the device image.
//
// The device image is organised for the kernels of pj_kernels.cu:
//   * reactions are sorted by class (pressure dependence, falloff form, reversibility) so that the
//     32 reactions a warp evaluates together take the same branches;
//   * every reaction owns "b-slots", one per species l whose mass-fraction column the reaction
//     touches directly (its reactants, products, non-unity third-body species, species m); the
//     kernel writes b'_il = c_i dR_i/d[X_l] + (dc_i/d[M]) R_i eps_il into them;
//   * static gather lists (CSR) turn the per-reaction terms into per-species sums without atomics:
//     species -> (reaction, nu) for the production rates and the dense coefficients, column ->
//     b-slots for the energy row, and (row k, column l) -> (b-slot, nu_ki) for the sparse block.
// The derivation of these terms from the paper's Section 3 chain rule is given in pj_kernels.cu.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <numeric>
#include <stdexcept>
#include <string>
#include <utility>
#include <vector>

#include "pj_internal.h"

namespace pj {

namespace {

struct Reader {
    const unsigned char *p, *end;
    template <class T> T get() {
        if (size_t(end - p) < sizeof(T)) throw FormatError("model buffer truncated");
        T v;
        std::memcpy(&v, p, sizeof(T));
        p += sizeof(T);
        return v;
    }
    int i32() { return get<int32_t>(); }
    double f64() { return get<double>(); }
};

struct HRxn {
    int kind = 0, rev = 0;
    std::vector<std::pair<int, int>> reac, prod;
    double A = 0, beta = 0, Ta = 0;
    double Ar = 0, betar = 0, Tar = 0;
    int tbmode = 0, tbsp = -1;
    std::vector<std::pair<int, double>> eff;      // alpha for listed species
    double k0[3] = {0, 0, 0}, ki[3] = {0, 0, 0};
    int ftype = 0, hasT2 = 0;
    double fp[5] = {0, 0, 0, 0, 0};
    std::vector<double> plog;                     // n x (p, A, beta, Ta)
    int nt = 0, npc = 0;
    double crng[4] = {0, 0, 0, 0};
    std::vector<double> eta;
};

struct HModel {
    int NE = 0, N = 0, R = 0;
    std::vector<double> W, Tmid, alo, ahi;
    std::vector<HRxn> rx;
};

void check(bool ok, const char *msg) {
    if (!ok) throw FormatError(msg);
}

HModel parse(const void *buf, size_t len) {
    Reader r{static_cast<const unsigned char *>(buf), static_cast<const unsigned char *>(buf) + len};
    char magic[8];
    for (char &c : magic) c = r.get<char>();
    check(std::memcmp(magic, "PYJACMEC", 8) == 0, "bad magic");
    uint32_t ver = r.get<uint32_t>(), ne = r.get<uint32_t>(), ns = r.get<uint32_t>(), nr = r.get<uint32_t>();
    check(ver == 1, "unsupported model format version");
    check(ns >= 2 && ns <= 30000 && nr <= 2000000 && ne <= 64, "model sizes out of range");
    HModel m;
    m.NE = int(ne);
    m.N = int(ns);
    m.R = int(nr);
    m.W.resize(ns);
    m.Tmid.resize(ns);
    m.alo.resize(7 * ns);
    m.ahi.resize(7 * ns);
    for (uint32_t k = 0; k < ns; ++k) {
        m.W[k] = r.f64();
        (void)r.f64();
        m.Tmid[k] = r.f64();
        (void)r.f64();
        for (int c = 0; c < 7; ++c) m.alo[7 * k + c] = r.f64();
        for (int c = 0; c < 7; ++c) m.ahi[7 * k + c] = r.f64();
        for (uint32_t e = 0; e < ne; ++e) (void)r.i32();
        check(m.W[k] > 0.0 && std::isfinite(m.W[k]), "species molecular weight must be positive");
    }
    m.rx.resize(nr);
    for (uint32_t i = 0; i < nr; ++i) {
        HRxn &x = m.rx[i];
        x.kind = r.i32();
        x.rev = r.i32();
        check(x.kind >= 0 && x.kind <= 5 && x.rev >= 0 && x.rev <= 2, "bad reaction kind or reversibility");
        for (int side = 0; side < 2; ++side) {
            int n = r.i32();
            check(n >= 0 && n <= 8, "too many species on one side of a reaction");
            auto &v = side ? x.prod : x.reac;
            for (int s = 0; s < n; ++s) {
                int sp = r.i32(), nu = r.i32();
                check(sp >= 0 && sp < int(ns) && nu >= 1 && nu <= 8, "bad stoichiometry entry");
                v.emplace_back(sp, nu);
            }
        }
        x.A = r.f64();
        x.beta = r.f64();
        x.Ta = r.f64();
        if (x.rev == kRevExplicit) {
            x.Ar = r.f64();
            x.betar = r.f64();
            x.Tar = r.f64();
        }
        if (x.kind == kThird || x.kind == kFalloff || x.kind == kChem) {
            x.tbmode = r.i32();
            x.tbsp = r.i32();
            int neff = r.i32();
            check(x.tbmode == kTbMix || x.tbmode == kTbSpecies, "bad third-body mode");
            check(x.tbmode != kTbSpecies || (x.tbsp >= 0 && x.tbsp < int(ns)), "bad third-body species");
            check(neff >= 0 && neff <= int(ns) && (neff == 0 || x.tbmode == kTbMix), "bad efficiency list");
            for (int e = 0; e < neff; ++e) {
                int sp = r.i32();
                double a = r.f64();
                check(sp >= 0 && sp < int(ns), "bad efficiency species");
                x.eff.emplace_back(sp, a);
            }
        }
        if (x.kind == kFalloff || x.kind == kChem) {
            for (double &v : x.k0) v = r.f64();
            for (double &v : x.ki) v = r.f64();
            x.ftype = r.i32();
            for (double &v : x.fp) v = r.f64();
            x.hasT2 = r.i32();
            check(x.ftype >= 0 && x.ftype <= 2, "bad falloff form");
        }
        if (x.kind == kPlog) {
            int n = r.i32();
            check(n >= 1 && n <= 64, "bad PLOG table size");
            x.plog.resize(4 * n);
            for (double &v : x.plog) v = r.f64();
            for (int c = 1; c < n; ++c) check(x.plog[4 * c] > x.plog[4 * (c - 1)], "PLOG pressures must increase");
            for (int c = 0; c < n; ++c) check(x.plog[4 * c] > 0 && x.plog[4 * c + 1] > 0, "PLOG p and A must be positive");
        }
        if (x.kind == kCheb) {
            x.nt = r.i32();
            x.npc = r.i32();
            check(x.nt >= 1 && x.npc >= 1 && x.nt <= 16 && x.npc <= 16, "bad Chebyshev shape");
            for (double &v : x.crng) v = r.f64();
            check(x.crng[0] > 0 && x.crng[1] > x.crng[0] && x.crng[2] > 0 && x.crng[3] > x.crng[2],
                  "bad Chebyshev range");
            x.eta.resize(size_t(x.nt) * x.npc);
            for (double &v : x.eta) v = r.f64();
        }
    }
    check(r.p == r.end, "trailing bytes after the last reaction");
    return m;
}

// Merge repeated species of one side into distinct (species, nu) slots.
std::vector<std::pair<int, int>> distinct(const std::vector<std::pair<int, int>> &v) {
    std::vector<std::pair<int, int>> out;
    for (auto &e : v) {
        bool found = false;
        for (auto &o : out)
            if (o.first == e.first) {
                o.second += e.second;
                found = true;
            }
        if (!found) out.push_back(e);
    }
    return out;
}

int class_key(const HRxn &x) {
    // The 32 reactions of a warp should take the same branches. Order: family (falloff and
    // chemically activated together, PLOG, Chebyshev, third-body, elementary), then falloff form
    // (a Troe falloff and a Troe chemically activated reaction share the F_cent / F work), kind,
    // third-body mode, reversibility, the number of distinct species on each side and whether all
    // of a side's coefficients are 1 (the shorter product code of side<UNIT>). The
    // cheapest family comes last, so the partly filled last round of a state runs the cheapest
    // code path (measured on B300: -7% FP64 instructions on a 53-species model).
    auto ndist = [](const std::vector<std::pair<int, int>> &v) {
        std::vector<int> s;
        for (auto &e : v)
            if (std::find(s.begin(), s.end(), e.first) == s.end()) s.push_back(e.first);
        return int(s.size());
    };
    const int fam = (x.kind == kFalloff || x.kind == kChem) ? 0
                    : x.kind == kPlog ? 1 : x.kind == kCheb ? 2 : x.kind == kThird ? 3 : 4;
    auto unit = [](const std::vector<std::pair<int, int>> &v) {
        for (auto &e : v)
            if (e.second != 1) return 0;
        return 1;
    };
    return ((((((fam * 4 + x.ftype) * 8 + x.kind) * 4 + x.tbmode) * 4 + x.rev) * 8 + ndist(x.reac)) * 8 +
            ndist(x.prod)) * 4 + unit(distinct(x.reac)) * 2 + unit(distinct(x.prod));
}

}  // namespace

namespace {

// One finished sum of a schedule: items (index, coefficient code, optional aux) summed in order
// by a single lane, then written to dst (with scale).
struct Task {
    std::vector<unsigned> idx;
    std::vector<int> code;
    std::vector<int> aux;
    int dst = 0;
    double scale = 0.0;
    bool partial = false;   // a later piece of a split row entry: sums from zero into partial slot dst
};

// Record layouts of the lane-balanced schedules.
enum RecMode {
    kRecPlain = 0,   // 2 words: item word (index | code << 24 | end << 31), destination on the last item
    kRecAux = 1,     // 4 words: item word, destination on the last item, aux value, 0
    kRecCoef = 2,    // 4 words: index | partial << 29 | first << 30 | end << 31, destination on every
                     // item, and the item's coefficient scale * nu as a double (the task's scale
                     // folded in)
};

// Lays out one chunk of tasks over the 32 lanes of a warp. Tasks are packed largest first onto
// the least-loaded lane (longest-processing-time rule); each lane's items run back to back with an
// end flag on the last item of every task; shorter lanes are padded with neutral items. Which lane
// evaluates a task does not change its value: a task is always summed by one lane, in the order
// its items are laid out here.
//
// Item order (shared-memory banks): the items of one record row are read by one load instruction
// per operand array, 32 lanes at once. A 64-bit load is served in half-warps; two lanes of a
// half-warp whose different indices agree mod 16 fall in the same pair of 4-byte banks and
// serialise. So the rows are filled one at a time, and each lane takes, of the items it may take
// next (the rest of its current task, or any item of a task it has not started), the first whose
// indices (the operand index, and for column sums also the reaction index) are free mod 16 in its
// half-warp so far; failing that, the one with the fewest clashes. The order depends on the model
// only, so every launch shape sums each task in the same order (bitwise the same results).
//
// Records are lane-interleaved (record ioff + 32 t + lane is the lane's t-th item). The chunk table
// gets (ioff, rows).
void emit_chunk(std::vector<const Task *> tasks, unsigned pad_idx, int pad_code, int pad_aux, RecMode mode,
                std::vector<uint32_t> &recs, std::vector<int> &chunk) {
    const int words = mode == kRecPlain ? 2 : 4;
    std::stable_sort(tasks.begin(), tasks.end(),
                     [](const Task *a, const Task *b) { return a->idx.size() > b->idx.size(); });
    std::vector<std::vector<const Task *>> lane(32);
    std::vector<size_t> load(32, 0);
    for (const Task *t : tasks) {
        int best = 0;
        for (int l = 1; l < 32; ++l)
            if (load[l] < load[best]) best = l;
        lane[best].push_back(t);
        load[best] += t->idx.size();
    }
    size_t len = 0;
    for (int l = 0; l < 32; ++l) len = std::max(len, load[l]);

    // bank-aware item order: seq[l][pos] = (task, item) or (null, 0) for a neutral item
    struct Slot {
        const Task *t = nullptr;
        int q = 0;
    };
    std::vector<std::vector<Slot>> seq(32, std::vector<Slot>(len));
    {
        struct LaneState {
            std::vector<const Task *> pending;   // tasks not started, in packing order
            const Task *cur = nullptr;
            std::vector<int> rest;               // items of cur not yet placed, in task order
        };
        std::vector<LaneState> ls(32);
        for (int l = 0; l < 32; ++l) ls[l].pending = lane[l];
        const bool two = mode == kRecAux;
        auto key0 = [&](const Slot &x) -> long long { return x.t ? (long long)x.t->idx[x.q] : (long long)pad_idx; };
        auto key1 = [&](const Slot &x) -> long long { return x.t ? (long long)x.t->aux[x.q] : (long long)pad_aux; };
        for (size_t row = 0; row < len; ++row) {
            for (int h = 0; h < 2; ++h) {
                // candidates of each lane of the half-warp (its next items), then a matching of lanes
                // to distinct banks (augmenting paths, lanes with the fewest choices first); a lane
                // left unmatched takes its candidate with the fewest clashes
                std::vector<std::vector<Slot>> cand(16);
                std::vector<int> start_task(16, -1);   // a lane starting a task: candidates from pending
                for (int i = 0; i < 16; ++i) {
                    LaneState &st = ls[16 * h + i];
                    if (st.cur && !st.rest.empty()) {
                        for (int u : st.rest) cand[i].push_back(Slot{st.cur, u});
                    } else if (!st.pending.empty()) {
                        start_task[i] = 1;
                        for (const Task *t : st.pending)
                            for (int u = 0; u < int(t->idx.size()); ++u) cand[i].push_back(Slot{t, u});
                    }
                }
                long long owner_addr[16];
                int owner[16];
                for (int b2 = 0; b2 < 16; ++b2) owner[b2] = -1, owner_addr[b2] = -1;
                bool pads = false;
                for (int i = 0; i < 16; ++i)
                    if (cand[i].empty()) pads = true;
                if (pads) {
                    owner[pad_idx & 15] = 16;              // the neutral items' shared address
                    owner_addr[pad_idx & 15] = pad_idx;
                }
                std::vector<int> choice(16, -1);
                std::vector<int> order;
                for (int i = 0; i < 16; ++i)
                    if (!cand[i].empty()) order.push_back(i);
                std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cand[x].size() < cand[y].size(); });
                std::function<bool(int, std::vector<char> &)> augment = [&](int i, std::vector<char> &seen) {
                    for (int c = 0; c < int(cand[i].size()); ++c) {
                        const long long a = key0(cand[i][c]);
                        const int bk = int(a & 15);
                        if (seen[bk] || owner[bk] == 16) continue;
                        seen[bk] = 1;
                        if (owner[bk] == -1 || augment(owner[bk], seen)) {
                            owner[bk] = i, owner_addr[bk] = a, choice[i] = c;
                            return true;
                        }
                    }
                    return false;
                };
                for (int i : order) {
                    std::vector<char> seen(16, 0);
                    augment(i, seen);
                }
                // unmatched lanes: the candidate with the fewest clashes against what the row holds so
                // far (an address already in the row costs nothing: the lanes share it); the column
                // sums' reaction index counts as a second operand
                std::vector<std::vector<long long>> in0(16), in1(16);
                auto add = [](std::vector<long long> &v, long long x) {
                    if (std::find(v.begin(), v.end(), x) == v.end()) v.push_back(x);
                };
                auto clash = [](const std::vector<long long> &v, long long x) {
                    return std::find(v.begin(), v.end(), x) != v.end() ? 0 : int(v.size());
                };
                if (pads) add(in1[pad_aux & 15], pad_aux);
                for (int b2 = 0; b2 < 16; ++b2)
                    if (owner[b2] != -1) add(in0[b2], owner_addr[b2]);
                if (two)
                    for (int i = 0; i < 16; ++i)
                        if (choice[i] >= 0) add(in1[key1(cand[i][choice[i]]) & 15], key1(cand[i][choice[i]]));
                for (int i : order) {
                    if (choice[i] >= 0) continue;
                    int bc = 1 << 30, bi = 0;
                    for (int c = 0; c < int(cand[i].size()) && bc > 0; ++c) {
                        int v = clash(in0[key0(cand[i][c]) & 15], key0(cand[i][c]));
                        if (two) v += clash(in1[key1(cand[i][c]) & 15], key1(cand[i][c]));
                        if (v < bc) bc = v, bi = c;
                    }
                    choice[i] = bi;
                    add(in0[key0(cand[i][bi]) & 15], key0(cand[i][bi]));
                    if (two) add(in1[key1(cand[i][bi]) & 15], key1(cand[i][bi]));
                }
                for (int i = 0; i < 16; ++i) {
                    const int l = 16 * h + i;
                    LaneState &st = ls[l];
                    if (choice[i] < 0) {
                        seq[l][row] = Slot{};
                        continue;
                    }
                    const Slot pick = cand[i][choice[i]];
                    if (start_task[i] >= 0) {
                        st.cur = pick.t;
                        st.pending.erase(std::find(st.pending.begin(), st.pending.end(), pick.t));
                        st.rest.clear();
                        for (int u = 0; u < int(pick.t->idx.size()); ++u)
                            if (u != pick.q) st.rest.push_back(u);
                    } else {
                        st.rest.erase(std::find(st.rest.begin(), st.rest.end(), pick.q));
                    }
                    seq[l][row] = pick;
                }
            }
        }
    }

    const size_t ioff = recs.size() / words;
    recs.resize((ioff + len * 32) * words, 0u);
    for (size_t x = ioff; x < ioff + len * 32; ++x) {           // neutral items (coefficient 0)
        recs[x * words] = mode == kRecCoef ? pad_idx : pad_idx | (unsigned(pad_code) << 24);
        if (mode == kRecAux) recs[x * words + 2] = uint32_t(pad_aux);
    }
    for (int l = 0; l < 32; ++l) {
        for (size_t pos = 0; pos < len; ++pos) {
            const Slot &x = seq[l][pos];
            if (!x.t) continue;
            const Task *t = x.t;
            const bool first = pos == 0 || seq[l][pos - 1].t != t;
            const bool last = pos + 1 == len || seq[l][pos + 1].t != t;
            uint32_t *r = &recs[(ioff + pos * 32 + l) * words];
            const unsigned end = last ? 0x80000000u : 0u;
            const int q = x.q;
            if (mode == kRecCoef) {
                r[0] = t->idx[q] | (first ? 0x40000000u : 0u) | (t->partial ? 0x20000000u : 0u) | end;
                r[1] = uint32_t(t->dst);
                const double coef = t->scale * double(t->code[q] - kNuBias);
                uint64_t bits;
                std::memcpy(&bits, &coef, 8);
                r[2] = uint32_t(bits);
                r[3] = uint32_t(bits >> 32);
            } else {
                r[0] = t->idx[q] | (unsigned(t->code[q]) << 24) | end;
                r[1] = last ? uint32_t(t->dst) : 0u;
                if (mode == kRecAux) r[2] = uint32_t(t->aux[q]);
            }
        }
    }
    chunk.push_back(int(ioff));
    chunk.push_back(int(len));
}

// A task with no items still has to write its (zero) result: give it one neutral item.
void ensure_nonempty(Task &t, unsigned pad_idx, int pad_code, int pad_aux) {
    if (t.idx.empty()) {
        t.idx.push_back(pad_idx);
        t.code.push_back(pad_code);
        t.aux.push_back(pad_aux);
    }
}

// Splits tasks into chunks with at least 32 x (longest task) items each, so that the longest
// task does not dominate its chunk, and at most n_max chunks; returns the chunks' task lists
// (balanced by item count).
std::vector<std::vector<const Task *>> split_chunks(const std::vector<Task> &tasks, int n_max = 16) {
    size_t total = 0, longest = 1;
    for (auto &t : tasks) {
        total += t.idx.size();
        longest = std::max(longest, t.idx.size());
    }
    int n = int(std::max<size_t>(1, (total + 32 * longest - 1) / (32 * longest)));
    n = std::min(n, n_max);
    std::vector<std::vector<const Task *>> out(n);
    std::vector<size_t> load(n, 0);
    std::vector<const Task *> order;
    for (auto &t : tasks) order.push_back(&t);
    std::stable_sort(order.begin(), order.end(),
                     [](const Task *a, const Task *b) { return a->idx.size() > b->idx.size(); });
    for (const Task *t : order) {
        int best = 0;
        for (int c = 1; c < n; ++c)
            if (load[c] < load[best]) best = c;
        out[best].push_back(t);
        load[best] += t->idx.size();
    }
    return out;
}

// Cuts every task into consecutive pieces of at most piece_len items (each piece one lane's
// ordered partial sum, written to partial slot dst = piece id). first[k] .. first[k+1] are the
// pieces of task k, in order.
std::vector<Task> cut_pieces(const std::vector<Task> &tasks, size_t piece_len, std::vector<int> &first) {
    std::vector<Task> out;
    first.assign(tasks.size() + 1, 0);
    for (size_t k = 0; k < tasks.size(); ++k) {
        first[k] = int(out.size());
        const Task &t = tasks[k];
        for (size_t b = 0; b < t.idx.size(); b += piece_len) {
            Task p;
            const size_t e = std::min(t.idx.size(), b + piece_len);
            p.idx.assign(t.idx.begin() + b, t.idx.begin() + e);
            p.code.assign(t.code.begin() + b, t.code.begin() + e);
            p.aux.assign(t.aux.begin() + b, t.aux.begin() + e);
            p.dst = int(out.size());
            p.scale = t.scale;
            out.push_back(std::move(p));
        }
    }
    first[tasks.size()] = int(out.size());
    return out;
}

// Piece length that lets the gather lists spread over n_warps warps of 32 lanes (at least 2
// items, so that a piece is never shorter than the combine step it adds).
size_t piece_length(const std::vector<Task> &tasks, int n_warps) {
    size_t total = 0;
    for (auto &t : tasks) total += t.idx.size();
    return std::max<size_t>(2, (total + 32 * size_t(n_warps) - 1) / (32 * size_t(n_warps)));
}

int nu_code(double nu) {
    const int v = int(nu);
    if (double(v) != nu || v < -kNuBias || v >= kNuBias) throw Unsupported("net stoichiometric coefficient out of range");
    return v + kNuBias;
}

}  // namespace

// Builds the host copy of the device image. Device pointers are patched by the caller.
HostImage build_image(const void *buf, size_t len) {
    HModel m = parse(buf, len);
    HostImage im;
    const int N = m.N, R = m.R;
    im.N = N;
    im.R = R;
    im.NE = m.NE;
    if (N > 32000) throw Unsupported("more than 32000 species");

    // species tables
    im.W = m.W;
    im.Tmid = m.Tmid;
    im.invW.resize(N);
    im.Delta.resize(N);
    for (int k = 0; k < N; ++k) im.invW[k] = 1.0 / m.W[k];
    for (int k = 0; k < N; ++k) im.Delta[k] = (k == N - 1) ? 0.0 : (1.0 / m.W[k] - 1.0 / m.W[N - 1]);
    im.thermo.assign(size_t(N) * kThermoStride, 0.0);
    for (int k = 0; k < N; ++k)
        for (int rng = 0; rng < 2; ++rng) {
            const double *a = rng ? &m.ahi[7 * k] : &m.alo[7 * k];
            double *t = &im.thermo[size_t(k) * kThermoStride + 18 * rng];
            for (int c = 0; c < 7; ++c) t[c] = a[c];
            t[7] = a[1] / 2.0;   // enthalpy and B_k / dB_k/dT coefficients
            t[8] = a[2] / 3.0;
            t[9] = a[3] / 4.0;
            t[10] = a[4] / 5.0;
            t[11] = a[2] / 6.0;
            t[12] = a[3] / 12.0;
            t[13] = a[4] / 20.0;
            t[14] = 2.0 * a[2];  // d(cp/R)/dT coefficients
            t[15] = 3.0 * a[3];
            t[16] = 4.0 * a[4];
            t[17] = a[6] - a[0];
        }

    // reaction order
    im.perm.resize(R);
    std::iota(im.perm.begin(), im.perm.end(), 0);
    std::stable_sort(im.perm.begin(), im.perm.end(),
                     [&](int a, int b) { return class_key(m.rx[a]) < class_key(m.rx[b]); });

    // per-reaction records, parameter pool, b-slots
    std::vector<std::vector<std::pair<int, double>>> net(R);   // sorted index -> (species, nu)
    std::vector<std::vector<int>> slot_species(R);
    im.rx.resize(R);
    int slot_total = 0;
    for (int si = 0; si < R; ++si) {
        const HRxn &x = m.rx[im.perm[si]];
        RxnDev d{};
        d.kind = uint8_t(x.kind);
        d.rev = uint8_t(x.rev);
        d.ftype = uint8_t(x.ftype);
        d.tbmode = uint8_t(x.kind == kThird || x.kind == kFalloff || x.kind == kChem ? x.tbmode : kTbNone);
        auto reac = distinct(x.reac), prod = distinct(x.prod);
        if (reac.size() > size_t(kMaxSlots) || prod.size() > size_t(kMaxSlots))
            throw Unsupported("more than 4 distinct species on one side of a reaction");
        d.nr = uint8_t(reac.size());
        d.np = uint8_t(prod.size());
        for (int s = 0; s < kMaxSlots; ++s) {
            d.rsp[s] = int16_t(s < d.nr ? reac[s].first : 0);
            d.rnu[s] = int8_t(s < d.nr ? reac[s].second : 0);
            d.psp[s] = int16_t(s < d.np ? prod[s].first : 0);
            d.pnu[s] = int8_t(s < d.np ? prod[s].second : 0);
        }
        for (auto &e : reac)
            if (e.second > kMaxNu) throw Unsupported("stoichiometric coefficient above 4");
        for (auto &e : prod)
            if (e.second > kMaxNu) throw Unsupported("stoichiometric coefficient above 4");
        auto all_unit = [](const std::vector<std::pair<int, int>> &v) {
            for (auto &e : v)
                if (e.second != 1) return false;
            return true;
        };
        d.flags = uint8_t((x.hasT2 ? 1 : 0) | (all_unit(reac) ? 2 : 0) | (all_unit(prod) ? 4 : 0));
        d.tbsp = int16_t(d.tbmode == kTbSpecies ? x.tbsp : 0);
        d.kform = kKfGeneral;
        d.kpow = 0;
        // parameter pool
        d.par_off = int(im.par.size());
        auto lnA = [](double A) {
            if (!(A > 0.0)) throw FormatError("Arrhenius prefactors must be positive");
            return std::log(A);
        };
        if (x.kind == kElem || x.kind == kThird) {
            im.par.insert(im.par.end(), {lnA(x.A), x.beta, x.Ta, x.A});
            if (x.beta == 0.0 && x.Ta == 0.0) d.kform = kKfConst;
            else if (x.Ta == 0.0 && x.beta == std::floor(x.beta) && std::fabs(x.beta) <= 4.0) {
                d.kform = kKfIntPow;
                d.kpow = int(x.beta);
            }
        } else if (x.kind == kFalloff || x.kind == kChem) {
            im.par.insert(im.par.end(), {lnA(x.k0[0]), x.k0[1], x.k0[2], lnA(x.ki[0]), x.ki[1], x.ki[2]});
            if (x.ftype == kTroe) {
                if (!(x.fp[1] > 0 && x.fp[2] > 0)) throw FormatError("Troe T*** and T* must be positive");
                im.par.insert(im.par.end(), {x.fp[0], 1.0 / x.fp[1], 1.0 / x.fp[2], x.fp[3], 0.0});
            } else if (x.ftype == kSri) {
                if (!(x.fp[2] > 0 && x.fp[3] > 0)) throw FormatError("SRI c and d must be positive");
                im.par.insert(im.par.end(), {x.fp[0], x.fp[1], 1.0 / x.fp[2], std::log(x.fp[3]), x.fp[4]});
            } else {
                im.par.insert(im.par.end(), {0.0, 0.0, 0.0, 0.0, 0.0});
            }
        } else if (x.kind == kPlog) {
            int n = int(x.plog.size() / 4);
            im.par.push_back(double(n));
            for (int c = 0; c < n; ++c)
                im.par.insert(im.par.end(), {x.plog[4 * c], std::log(x.plog[4 * c]), lnA(x.plog[4 * c + 1]),
                                             x.plog[4 * c + 2], x.plog[4 * c + 3]});
        } else {   // Chebyshev
            double Tsum = 1.0 / x.crng[0] + 1.0 / x.crng[1];
            double Tscale = 1.0 / (1.0 / x.crng[1] - 1.0 / x.crng[0]);
            double lPsum = std::log10(x.crng[2]) + std::log10(x.crng[3]);
            double lPscale = 1.0 / (std::log10(x.crng[3]) - std::log10(x.crng[2]));
            im.par.insert(im.par.end(), {double(x.nt), double(x.npc), Tsum, Tscale, lPsum, lPscale});
            im.par.insert(im.par.end(), x.eta.begin(), x.eta.end());
        }
        if (x.rev == kRevExplicit) im.par.insert(im.par.end(), {lnA(x.Ar), x.betar, x.Tar});

        // third-body efficiencies (mixture): epsilon = alpha - 1 for listed species, merged
        std::map<int, double> eps;
        if (d.tbmode == kTbMix)
            for (auto &e : x.eff) eps[e.first] = e.second - 1.0;
        d.eff_off = int(im.eff_sp.size());
        int neff = 0;
        for (auto &e : eps)
            if (e.second != 0.0) {
                im.eff_sp.push_back(e.first);
                im.eff_eps.push_back(e.second);
                ++neff;
            }
        d.neff = int16_t(neff);

        // b-slots: reactants, products, non-unity efficiency species, species m
        std::vector<int> sl;
        auto add = [&](int sp) {
            if (std::find(sl.begin(), sl.end(), sp) == sl.end()) sl.push_back(sp);
        };
        for (auto &e : reac) add(e.first);
        for (auto &e : prod) add(e.first);
        if (d.tbmode == kTbMix && (x.kind == kThird || x.kind == kFalloff || x.kind == kChem))
            for (auto &e : eps)
                if (e.second != 0.0) add(e.first);
        if (d.tbmode == kTbSpecies) add(x.tbsp);
        d.slot_off = slot_total;
        d.nslot = int(sl.size());
        for (int sp : sl) {
            int rs = -1, ps = -1;
            for (int s = 0; s < d.nr; ++s)
                if (reac[s].first == sp) rs = s;
            for (int s = 0; s < d.np; ++s)
                if (prod[s].first == sp) ps = s;
            double e = 0.0;
            if (d.tbmode == kTbMix) {
                auto it = eps.find(sp);
                if (it != eps.end()) e = it->second;
            } else if (d.tbmode == kTbSpecies) {
                e = (sp == x.tbsp) ? 1.0 : 0.0;
            }
            im.slot_info.push_back(sp | ((rs + 1) << 16) | ((ps + 1) << 24));
            im.slot_eps.push_back(e);
        }
        slot_species[si] = sl;
        slot_total += d.nslot;
        // net stoichiometry
        std::map<int, int> nn;
        for (auto &e : reac) nn[e.first] -= e.second;
        for (auto &e : prod) nn[e.first] += e.second;
        for (auto &e : nn)
            if (e.second != 0) net[si].emplace_back(e.first, double(e.second));
        im.rx[si] = d;
    }

    // species gather CSR: species k -> (reaction, nu_ki), reactions ascending
    {
        std::vector<std::vector<std::pair<int, double>>> lists(N);
        for (int i = 0; i < R; ++i)
            for (auto &e : net[i]) lists[e.first].emplace_back(i, e.second);
        im.sp_ptr.assign(N + 1, 0);
        for (int k = 0; k < N; ++k) {
            im.sp_ptr[k + 1] = im.sp_ptr[k] + int(lists[k].size());
            for (auto &e : lists[k]) {
                im.sp_rxn.push_back(e.first);
                im.sp_nu.push_back(e.second);
            }
        }
    }
    // energy-row column CSR: column l -> b-slots (reaction ascending)
    {
        std::vector<std::vector<std::pair<int, int>>> lists(N);
        for (int i = 0; i < R; ++i)
            for (int s = 0; s < int(slot_species[i].size()); ++s)
                lists[slot_species[i][s]].emplace_back(im.rx[i].slot_off + s, i);
        im.col_ptr.assign(N + 1, 0);
        for (int l = 0; l < N; ++l) {
            im.col_ptr[l + 1] = im.col_ptr[l] + int(lists[l].size());
            for (auto &e : lists[l]) {
                im.col_slot.push_back(e.first);
                im.col_rxn.push_back(e.second);
            }
        }
    }
    // sparse block: (row k, column l) -> contributions (b-slot of reaction i for l, nu_ki)
    {
        std::map<std::pair<int, int>, std::vector<std::pair<int, double>>> pairs;
        for (int i = 0; i < R; ++i)
            for (auto &e : net[i])
                for (int s = 0; s < int(slot_species[i].size()); ++s)
                    pairs[{e.first, slot_species[i][s]}].emplace_back(im.rx[i].slot_off + s, e.second);
        im.row_ptr.assign(N + 1, 0);
        im.colN_nnz.assign(N, -1);
        im.nnz_cptr.push_back(0);
        for (auto &kv : pairs) {
            int k = kv.first.first, l = kv.first.second;
            int e = int(im.nnz_col.size());
            im.nnz_col.push_back(l);
            im.nnz_wr.push_back(m.W[k] / m.W[l]);
            for (auto &c : kv.second) {
                im.con_slot.push_back(c.first);
                im.con_nu.push_back(c.second);
            }
            im.nnz_cptr.push_back(int(im.con_slot.size()));
            im.row_ptr[k + 1]++;
            if (l == N - 1) im.colN_nnz[k] = e;
        }
        for (int k = 0; k < N; ++k) im.row_ptr[k + 1] += im.row_ptr[k];
    }
    // molar-concentration basis: species row k < N-1 holds the columns n_j (j < N-1) of its
    // sparse-block entries, or every column when its row has an entry in column N (d/dn_j moves
    // [X_N] by -1/V, so D_kN enters every column); ascending j
    {
        im.cc_ptr.assign(N, 0);
        for (int k = 0; k < N - 1; ++k) {
            const bool dense = im.colN_nnz[k] >= 0;
            std::vector<char> at(N - 1, 0);
            for (int e = im.row_ptr[k]; e < im.row_ptr[k + 1]; ++e)
                if (im.nnz_col[e] < N - 1) at[im.nnz_col[e]] = 1;
            for (int j = 0; j < N - 1; ++j)
                if (dense || at[j]) {
                    im.cc_col.push_back(j);
                    im.cc_wr.push_back(m.W[j] / m.W[k]);
                }
            im.cc_ptr[k + 1] = int(im.cc_col.size());
        }
        im.rx_dnu.assign(R + 1, 0.0);                 // + the zero that padded schedule items read
        for (int i = 0; i < R; ++i)
            for (auto &e : net[i]) im.rx_dnu[i] += e.second;
    }

    // lane-balanced schedules; neutral items read the zero element appended to each array
    const unsigned zero_slot = unsigned(slot_total), zero_rxn = unsigned(R);
    const int zero_code = kNuBias;   // nu = 0
    if (slot_total >= (1 << 24) || R >= (1 << 24)) throw Unsupported("more than 2^24 reactions or b-slots");
    // species gather: omega_k, J_k0, A_k from (reaction, nu_ki)
    {
        std::vector<Task> tasks(N);
        for (int k = 0; k < N; ++k) {
            tasks[k].dst = k;
            for (int e = im.sp_ptr[k]; e < im.sp_ptr[k + 1]; ++e) {
                tasks[k].idx.push_back(unsigned(im.sp_rxn[e]));
                tasks[k].code.push_back(nu_code(im.sp_nu[e]));
                tasks[k].aux.push_back(0);
            }
            ensure_nonempty(tasks[k], zero_rxn, zero_code, 0);
        }
        const int nw = default_wps(N, true);
        auto pieces = cut_pieces(tasks, piece_length(tasks, nw), im.g_pfirst);
        im.ngp = int(pieces.size());
        auto chunks = split_chunks(pieces, nw);
        for (auto &c : chunks) emit_chunk(c, zero_rxn, zero_code, 0, kRecPlain, im.g_rec, im.g_chunk);
        im.ng = int(chunks.size());
    }
    // energy-row column sums HS_j from (b-slot, reaction)
    {
        std::vector<Task> tasks(N);
        for (int l = 0; l < N; ++l) {
            tasks[l].dst = l;
            for (int e = im.col_ptr[l]; e < im.col_ptr[l + 1]; ++e) {
                tasks[l].idx.push_back(unsigned(im.col_slot[e]));
                tasks[l].code.push_back(zero_code);
                tasks[l].aux.push_back(im.col_rxn[e]);
            }
            ensure_nonempty(tasks[l], zero_slot, zero_code, R);
        }
        const int nw = default_wps(N, true);
        auto pieces = cut_pieces(tasks, piece_length(tasks, nw), im.h_pfirst);
        im.nhp = int(pieces.size());
        auto chunks = split_chunks(pieces, nw);
        for (auto &c : chunks)
            emit_chunk(c, zero_slot, zero_code, R, kRecAux, im.h_rec, im.h_chunk);
        im.nh = int(chunks.size());
    }
    // C_k = -(W_k/W_N) sum nu_ki b'_iN, from the sparse entries of column N-1 (cut into pieces
    // like the gathers above; a combine adds a species' pieces in order)
    {
        std::vector<Task> tasks(N);
        for (int k = 0; k < N; ++k) {
            tasks[k].dst = k;
            const int e = im.colN_nnz[k];
            if (e >= 0) {
                tasks[k].scale = -im.nnz_wr[e];   // C_k = -(W_k/W_N) sum ...
                for (int c = im.nnz_cptr[e]; c < im.nnz_cptr[e + 1]; ++c) {
                    tasks[k].idx.push_back(unsigned(im.con_slot[c]));
                    tasks[k].code.push_back(nu_code(im.con_nu[c]));
                    tasks[k].aux.push_back(0);
                }
            }
            ensure_nonempty(tasks[k], zero_slot, zero_code, 0);
        }
        const int nw = default_wps(N, true);
        auto pieces = cut_pieces(tasks, piece_length(tasks, nw), im.c_pfirst);
        im.ncp = int(pieces.size());
        auto chunks = split_chunks(pieces, nw);
        for (auto &c : chunks)
            emit_chunk(c, zero_slot, zero_code, 0, kRecCoef, im.c_rec, im.c_chunk);
        im.ncc = int(chunks.size());
    }
    // sparse block, per chunk of rpc staged rows (row r = species r-1, row 0 = energy row). A
    // chunk's lanes are balanced only if no entry is much longer than the chunk's items / 32, so
    // entries longer than that are cut into pieces: the first piece starts from the dense value
    // and ends in the staged row as before; each later piece sums from zero into a partial slot of
    // the warp, and a combine list adds an entry's partials to it in piece order.
    {
        im.rpc = std::max(1, std::min(4, 256 / (N + 1)));
        im.n_row_chunks = (N + 1 + im.rpc - 1) / im.rpc;
        im.s_npart = 0;
        for (int c = 0; c < im.n_row_chunks; ++c) {
            const int r0 = c * im.rpc, r1 = std::min(r0 + im.rpc, N + 1);
            std::vector<Task> tasks;
            size_t total = 0;
            for (int r = std::max(r0, 1); r < r1; ++r) {
                const int k = r - 1;
                for (int e = im.row_ptr[k]; e < im.row_ptr[k + 1]; ++e) {
                    const int j = im.nnz_col[e];
                    if (j == N - 1) continue;
                    Task t;
                    t.dst = (r - r0) * (N + 1) + 1 + j;
                    t.scale = im.nnz_wr[e];
                    for (int q = im.nnz_cptr[e]; q < im.nnz_cptr[e + 1]; ++q) {
                        t.idx.push_back(unsigned(im.con_slot[q]));
                        t.code.push_back(nu_code(im.con_nu[q]));
                        t.aux.push_back(0);
                    }
                    total += t.idx.size();
                    tasks.push_back(std::move(t));
                }
            }
            const size_t plen = std::max<size_t>(2, (total + 31) / 32);
            std::vector<Task> pieces;
            int npart = 0;
            std::vector<std::array<int, 3>> split;   // (staged position, first partial slot, partials)
            for (const Task &t : tasks) {
                const size_t n = t.idx.size();
                // at most 32 pieces, so that an entry's value and partials fit one warp's lanes
                const size_t len = std::max(plen, (n + 31) / 32);
                int first_part = -1, nparts = 0;
                for (size_t b = 0; b < n; b += len) {
                    Task p;
                    const size_t e = std::min(n, b + len);
                    for (size_t q = b; q < e; ++q) {
                        p.idx.push_back(t.idx[q]);
                        p.code.push_back(t.code[q]);
                        p.aux.push_back(t.aux[q]);
                    }
                    p.scale = t.scale;
                    if (b == 0) {
                        p.dst = t.dst;
                    } else {
                        p.partial = true;
                        p.dst = npart++;
                        if (first_part < 0) first_part = p.dst;
                        ++nparts;
                    }
                    pieces.push_back(std::move(p));
                }
                if (nparts > 0) split.push_back({t.dst, first_part, nparts});
            }
            // combine passes: the split entries' segments [staged value, partial 0, partial 1, ...]
            // packed onto the 32 lanes of a warp in entry order, each pass summed by a fixed pairwise
            // tree within every segment (levels: enough for the pass's longest segment)
            const int first_pass = int(im.s_comb.size() / 64);
            int npass = 0;
            for (size_t a = 0; a < split.size();) {
                size_t b = a;
                int lanes = 0, longest = 0;
                while (b < split.size() && lanes + split[b][2] + 1 <= 32) {
                    lanes += split[b][2] + 1;
                    longest = std::max(longest, split[b][2] + 1);
                    ++b;
                }
                int levels = 0;
                while ((1 << levels) < longest) ++levels;
                std::vector<int> rec(64, 0);
                int l = 0;
                for (size_t e = a; e < b; ++e) {
                    const int seg = split[e][2] + 1;
                    for (int q = 0; q < seg; ++q, ++l) {
                        rec[2 * l] = q == 0 ? split[e][0] : -1 - (split[e][1] + q - 1);
                        rec[2 * l + 1] = q | (seg << 8) | (levels << 16);
                    }
                }
                for (; l < 32; ++l) rec[2 * l + 1] = levels << 16;   // idle lanes (segment length 0)
                im.s_comb.insert(im.s_comb.end(), rec.begin(), rec.end());
                ++npass;
                a = b;
            }
            im.s_comb_chunk.push_back(first_pass);
            im.s_comb_chunk.push_back(npass);
            im.s_npart = std::max(im.s_npart, npart);
            std::vector<const Task *> ptrs;
            for (auto &t : pieces) ptrs.push_back(&t);
            emit_chunk(ptrs, zero_slot, zero_code, 0, kRecCoef, im.s_rec, im.s_chunk);
        }
        if (im.s_comb.empty()) im.s_comb.assign(64, 0);
    }
    return im;
}

}  // namespace pj
