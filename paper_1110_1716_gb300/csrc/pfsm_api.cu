// Host side of libpfsm: contexts, machine loading and residency, scans.
//
// A machine is validated and turned into its device encoding once, at load
// (Sec. III.A: the PFSM runs on the caller's unconverted DFA or NFA table;
// nothing is determinised or compacted). Device copies live under a byte
// budget with least-recently-used eviction and transparent reload: the
// device form of the paper's remedy for insomnia (Sec. I-II), where cold
// automata leave fast memory and come back when needed.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <map>
#include <mutex>
#include <vector>

#include "pfsm_host.h"

using namespace pfsm;

namespace pfsm {

int ceil_log2(int S) {
    int b = 0;
    while ((1 << b) < S) ++b;
    return std::max(1, b);
}

// Default depth of the start-prefix table: the k-gram index has k * sbits
// bits; the table holds 2^(k*sbits) uint16 entries (shared memory when it
// fits beside the rest, else L2). An NFA takes the deepest table (16 bits):
// every prefix step it covers is a set union the scan no longer performs
// per start (a record pool too large for 16-bit offsets lowers k at load).
// A DFA step is a single lookup: 12 bits keep its table and records small.
int default_k(const Machine &m) {
    if (m.sbits >= 8) return 2;
    const int max_bits = m.kind == 0 ? 12 : 16;   // 8 KB / 128 KB of entries
    int k = std::max(1, max_bits / m.sbits);
    return std::min(k, 8);
}

// ---- start-prefix table ---------------------------------------------------
// DFA: entry for k-gram w = outcome of stepping q0 through w.
void build_memo_dfa(Machine &m) {
    const int k = m.k;
    if (k <= 0) {
        m.memo.clear();
        return;
    }
    const uint32_t nent = 1u << (k * m.sbits);
    const uint32_t smask = (1u << m.sbits) - 1;
    m.memo.assign(nent + (nent & 1), PT_SKIP);
    m.pool.clear();
    std::map<std::vector<uint32_t>, uint32_t> recs;
    std::vector<uint32_t> matches, rec;
    for (uint32_t w = 0; w < nent; ++w) {
        int s = m.q0;
        bool died = false, bad = false;
        matches.clear();
        for (int j = 0; j < k; ++j) {
            const int a = (w >> (j * m.sbits)) & smask;
            if (a >= m.S) {
                bad = true;
                break;
            }
            const uint16_t e = m.dtab[(size_t)s * m.S + a];
            if (e == DEAD16) {
                died = true;
                break;
            }
            s = e & 0x7FFF;
            if (e & FINAL_BIT) matches.push_back((static_cast<uint32_t>(j) << 16) | static_cast<uint32_t>(s));
        }
        if (bad) continue;   // such k-grams raise E_INVAL anyway
        if (matches.empty()) {
            m.memo[w] = died ? PT_SKIP : static_cast<uint16_t>(s);
            continue;
        }
        // matches within the k steps: a record of them and the survivor
        rec.assign(1, static_cast<uint32_t>(matches.size()) | ((died ? 0u : 1u) << 16));
        rec.insert(rec.end(), matches.begin(), matches.end());
        if (!died) rec.push_back(static_cast<uint32_t>(s));
        auto it = recs.find(rec);
        uint32_t at;
        if (it != recs.end()) {
            at = it->second;
        } else {
            at = static_cast<uint32_t>(m.pool.size());
            if (at + rec.size() > PT_REC_MAX) {
                m.memo[w] = PT_WALK;   // the pool is full: step from q0 instead
                continue;
            }
            recs.emplace(rec, at);
            m.pool.insert(m.pool.end(), rec.begin(), rec.end());
        }
        m.memo[w] = static_cast<uint16_t>(PT_REC | at);
    }
    if (m.pool.empty()) m.pool.push_back(0);
}

// NFA: entry for k-gram w = record of the matches met within the first k
// steps from {q0} and the state set after them; equal records are shared.
// delta(q, a) of an NFA as uint16 entries (state | FINAL_BIT), each target
// followed by the states it reaches through epsilon edges when the machine
// keeps them (step 2 of Sec. III.B applied after every symbol).
template <class F>
static void nfa_step(const Machine &m, uint32_t q, int a, F &&f) {
    const uint32_t lo = m.off[(size_t)q * m.S + a], hi = m.off[(size_t)q * m.S + a + 1];
    for (uint32_t e = lo; e < hi; ++e) {
        const uint16_t t = m.tgt[e];
        f(t);
        if (!m.ecl_off.empty()) {
            const uint32_t ts = t & 0x7FFF;
            for (uint32_t x = m.ecl_off[ts]; x < m.ecl_off[ts + 1]; ++x) f(m.ecl_tgt[x]);
        }
    }
}

// The state set an instance starts with: q0 and what it reaches through
// epsilon edges (a final state among them reports nothing: no empty matches).
static std::vector<uint16_t> nfa_initial(const Machine &m) {
    std::vector<uint16_t> s{static_cast<uint16_t>(m.q0)};
    if (!m.ecl_off.empty())
        for (uint32_t x = m.ecl_off[m.q0]; x < m.ecl_off[m.q0 + 1]; ++x)
            s.push_back(static_cast<uint16_t>(m.ecl_tgt[x] & 0x7FFF));
    std::sort(s.begin(), s.end());
    s.erase(std::unique(s.begin(), s.end()), s.end());
    return s;
}

struct NfaMemoBuilder {
    Machine &m;
    std::map<std::vector<uint32_t>, uint32_t> recs, recs2;
    std::vector<uint32_t> mark;
    uint32_t stamp = 0;
    bool ok = true;
    // second level: the survivor sets of first-level records without
    // matches, indexed in order of appearance, and where their index words
    // sit in the pool
    bool l2 = false;
    std::map<std::vector<uint16_t>, uint32_t> set_index;
    std::vector<std::vector<uint16_t>> l2sets;
    std::vector<size_t> index_words;

    explicit NfaMemoBuilder(Machine &mm) : m(mm), mark(mm.Q, 0) {}

    static std::vector<uint32_t> encode(const std::vector<uint32_t> &matches,
                                        const std::vector<uint16_t> &set) {
        std::vector<uint32_t> rec;
        rec.push_back(static_cast<uint32_t>(matches.size()) |
                      (static_cast<uint32_t>(set.size()) << 16));
        rec.insert(rec.end(), matches.begin(), matches.end());
        for (uint16_t q : set) rec.push_back(q);
        return rec;
    }

    uint16_t record(const std::vector<uint32_t> &matches, const std::vector<uint16_t> &set) {
        std::vector<uint32_t> rec = encode(matches, set);
        const bool indexed = l2 && matches.empty() && !set.empty();
        if (indexed) {
            auto si = set_index.find(set);
            uint32_t x = static_cast<uint32_t>(l2sets.size());
            if (si == set_index.end()) {
                set_index.emplace(set, x);
                l2sets.push_back(set);
            } else {
                x = si->second;
            }
            rec.push_back(x < L2_MAX_SETS ? x : L2_NONE);
        }
        auto it = recs.find(rec);
        if (it != recs.end()) return static_cast<uint16_t>(it->second);
        const uint32_t at = static_cast<uint32_t>(m.pool.size());
        if (at >= PT_WALK || matches.size() > 0xFFFF || set.size() > 0xFFFF) {
            ok = false;
            return PT_SKIP;
        }
        recs.emplace(rec, at);
        m.pool.insert(m.pool.end(), rec.begin(), rec.end());
        if (indexed) index_words.push_back(m.pool.size() - 1);
        return static_cast<uint16_t>(at);
    }

    // second-level record: word offset in pool2, or L2_EMPTY (and ok2 false)
    // when pool2 is full
    bool ok2 = true;
    uint16_t record2(const std::vector<uint32_t> &matches, const std::vector<uint16_t> &set) {
        std::vector<uint32_t> rec = encode(matches, set);
        auto it = recs2.find(rec);
        if (it != recs2.end()) return static_cast<uint16_t>(it->second);
        const uint32_t at = static_cast<uint32_t>(m.pool2.size());
        if (at >= L2_EMPTY || matches.size() > 0xFFFF || set.size() > 0xFFFF) {
            ok2 = false;
            return L2_EMPTY;
        }
        recs2.emplace(rec, at);
        m.pool2.insert(m.pool2.end(), rec.begin(), rec.end());
        return static_cast<uint16_t>(at);
    }

    // One step of a set on symbol a: the next set (sorted) and the finals met,
    // recorded as (index of the symbol from the start) << 16 | state.
    void step(const std::vector<uint16_t> &set, int a, uint32_t sym_index,
              std::vector<uint16_t> &next, std::vector<uint32_t> &nm) {
        ++stamp;
        for (uint16_t q : set) {
            nfa_step(m, q, a, [&](uint16_t t) {
                const uint16_t ts = t & 0x7FFF;
                if (mark[ts] == stamp) return;
                mark[ts] = stamp;
                next.push_back(ts);
                if (t & FINAL_BIT) nm.push_back((sym_index << 16) | ts);
            });
        }
        std::sort(next.begin(), next.end());
    }

    // second level of set x: d of its L2_SYMS symbols consumed (g holds them)
    void dfs2(uint32_t x, int d, uint32_t g, const std::vector<uint16_t> &set,
              const std::vector<uint32_t> &matches) {
        if (!ok2) return;
        uint16_t *tab = m.l2tab.data() + static_cast<size_t>(x) * L2_GRAMS;
        if (d == L2_SYMS) {
            if (!matches.empty() || !set.empty()) tab[g] = record2(matches, set);
            return;
        }
        if (set.empty()) {
            // every extension of these d symbols has the same record
            if (matches.empty()) return;   // L2_EMPTY already
            const uint16_t id = record2(matches, set);
            for (uint32_t hiw = 0; hiw < (1u << (2 * (L2_SYMS - d))); ++hiw)
                tab[g | (hiw << (2 * d))] = id;
            return;
        }
        for (int a = 0; a < 4; ++a) {
            if (a >= m.S) continue;   // such grams raise E_INVAL anyway
            std::vector<uint16_t> next;
            std::vector<uint32_t> nm = matches;
            step(set, a, static_cast<uint32_t>(m.k + d), next, nm);
            dfs2(x, d + 1, g | (static_cast<uint32_t>(a) << (2 * d)), next, nm);
        }
    }

    // The second-level tables of the indexed sets; without them (too many
    // records) every index word becomes L2_NONE.
    void build_l2() {
        const uint32_t nsets = static_cast<uint32_t>(std::min<size_t>(l2sets.size(), L2_MAX_SETS));
        m.l2tab.assign(static_cast<size_t>(nsets) * L2_GRAMS, L2_EMPTY);
        m.pool2.clear();
        for (uint32_t x = 0; x < nsets && ok2; ++x) dfs2(x, 0, 0, l2sets[x], {});
        if (!ok2 || nsets == 0) {
            m.l2tab.clear();
            m.pool2.clear();
            for (size_t w : index_words) m.pool[w] = L2_NONE;
        }
    }

    // depth symbols consumed (index bits below depth*sbits fixed to prefix)
    void dfs(int depth, uint32_t prefix, const std::vector<uint16_t> &set,
             const std::vector<uint32_t> &matches) {
        if (!ok) return;
        const int k = m.k, sb = m.sbits;
        // a text that ends here: the matches so far are the start's result
        if (depth > 0 && depth < k && !matches.empty())
            m.tail[tail_base(depth, sb) + prefix] = record(matches, {});
        if (depth == k) {
            if (!matches.empty() || !set.empty()) m.memo[prefix] = record(matches, set);
            return;
        }
        if (set.empty()) {
            // nothing survives: every extension of this prefix has this record
            if (matches.empty()) return;
            const uint16_t id = record(matches, set);
            const uint32_t rest = static_cast<uint32_t>(k - depth) * sb;
            for (uint32_t hiw = 0; hiw < (1u << rest); ++hiw)
                m.memo[prefix | (hiw << (depth * sb))] = id;
            // and every longer short gram through this prefix
            for (int j = std::max(depth + 1, 1); j < k; ++j)
                for (uint32_t hiw = 0; hiw < (1u << ((j - depth) * sb)); ++hiw)
                    m.tail[tail_base(j, sb) + (prefix | (hiw << (depth * sb)))] = id;
            return;
        }
        for (int a = 0; a < (1 << sb); ++a) {
            if (a >= m.S) continue;   // such k-grams raise E_INVAL anyway
            std::vector<uint16_t> next;
            std::vector<uint32_t> nm = matches;
            step(set, a, static_cast<uint32_t>(depth), next, nm);
            dfs(depth + 1, prefix | (static_cast<uint32_t>(a) << (depth * sb)), next, nm);
        }
    }
};

bool build_memo_nfa(Machine &m) {
    m.pool.clear();
    m.tail.clear();
    m.l2tab.clear();
    m.pool2.clear();
    m.memox.clear();
    if (m.k <= 0) {
        m.memo.clear();
        return true;
    }
    const uint32_t nent = 1u << (m.k * m.sbits);
    m.memo.assign(nent + (nent & 1), PT_SKIP);
    const uint32_t ntail = tail_base(m.k, m.sbits);
    m.tail.assign(ntail + (ntail & 1), PT_SKIP);
    NfaMemoBuilder b(m);
    // second level where one packed 16-symbol gram covers k + L2_SYMS symbols
    b.l2 = m.sbits == 2 && m.k + L2_SYMS <= 16;
    b.dfs(0, 0, nfa_initial(m), {});
    if (!b.ok) return false;
    if (b.l2) b.build_l2();
    if (m.pool.empty()) m.pool.push_back(0);
    // the second-level set index of every k-gram's record, beside the table
    m.memox.clear();
    if (!m.l2tab.empty()) {
        m.memox.assign(m.memo.size(), L2_NONE);
        for (size_t g = 0; g < m.memo.size(); ++g) {
            const uint32_t e = m.memo[g];
            if (e >= PT_WALK) continue;
            const uint32_t hdr = m.pool[e];
            if ((hdr & 0xFFFFu) == 0 && (hdr >> 16) != 0)
                m.memox[g] = static_cast<uint16_t>(m.pool[e + 1 + (hdr >> 16)]);
        }
    }
    return true;
}

bool build_memo(Machine &m) {
    if (m.kind == 0) {
        build_memo_dfa(m);
        return true;
    }
    return build_memo_nfa(m);
}

// ---- survival bitmaps ---------------------------------------------------
// One bit per m-gram w (index sum_j w[j] << (j * sbits)): set when an instance
// started at q0 either reaches a final state within the m symbols of w or
// still holds a state after them. A clear bit proves that a start whose next
// m symbols are w reports nothing, so the filter drops it with one bit test.
// Built depth-first; a subtree is settled as soon as the set empties (all
// clear) or a final state is met (all set). Returns false (and no bitmap)
// when fewer than half of the m-grams are clear.
static bool survival_bits(const Machine &m, int mm, std::vector<uint32_t> &bits) {
    const uint32_t nbits = 1u << (mm * m.sbits);
    bits.assign((nbits + 31) / 32, 0);
    uint64_t ones = 0;
    auto set_range = [&](uint32_t p, int depth) {   // all extensions of a depth-long prefix
        const uint32_t rest = static_cast<uint32_t>(mm - depth) * m.sbits;
        for (uint32_t hw = 0; hw < (1u << rest); ++hw) {
            const uint32_t w = p | (hw << (depth * m.sbits));
            bits[w >> 5] |= 1u << (w & 31);
        }
        ones += 1ull << rest;
    };
    if (m.kind == 0) {
        std::function<void(int, uint32_t, int)> dfs = [&](int depth, uint32_t prefix, int s) {
            if (depth == mm) {
                bits[prefix >> 5] |= 1u << (prefix & 31);
                ++ones;
                return;
            }
            for (int a = 0; a < (1 << m.sbits) && a < m.S; ++a) {
                const uint16_t e = m.dtab[(size_t)s * m.S + a];
                if (e == DEAD16) continue;
                const uint32_t p = prefix | (static_cast<uint32_t>(a) << (depth * m.sbits));
                if (e & FINAL_BIT) set_range(p, depth + 1);
                else dfs(depth + 1, p, e & 0x7FFF);
            }
        };
        dfs(0, 0, m.q0);
    } else {
        std::vector<uint32_t> mark(m.Q, 0);
        uint32_t stamp = 0;
        std::vector<std::vector<uint16_t>> lv(mm + 1);
        std::function<void(int, uint32_t)> dfs = [&](int depth, uint32_t prefix) {
            const std::vector<uint16_t> &S = lv[depth];
            if (depth == mm) {
                bits[prefix >> 5] |= 1u << (prefix & 31);
                ++ones;
                return;
            }
            for (int a = 0; a < (1 << m.sbits) && a < m.S; ++a) {
                std::vector<uint16_t> &N = lv[depth + 1];
                N.clear();
                bool hit = false;
                ++stamp;
                for (uint16_t q : S) {
                    nfa_step(m, q, a, [&](uint16_t t) {
                        const uint16_t ts = t & 0x7FFF;
                        if (t & FINAL_BIT) hit = true;
                        if (mark[ts] == stamp) return;
                        mark[ts] = stamp;
                        N.push_back(ts);
                    });
                }
                const uint32_t p = prefix | (static_cast<uint32_t>(a) << (depth * m.sbits));
                if (hit) set_range(p, depth + 1);
                else if (!N.empty()) dfs(depth + 1, p);
            }
        };
        lv[0] = nfa_initial(m);
        dfs(0, 0);
    }
    if (ones * 2 > nbits) {
        bits.clear();
        return false;
    }
    return true;
}

// Two filters: a shallow one kept in shared memory (<= 32 KB) and a deep
// one read from global memory / L2 (<= 8 MB) for the starts that pass the
// first.

void build_survival(Machine &m) {
    m.surv.clear();
    m.surv2.clear();
    m.sm_m = 0;
    m.sm_m2 = 0;
    const int m1 = std::min(9, 18 / m.sbits);
    if (m1 >= 1 && survival_bits(m, m1, m.surv)) m.sm_m = m1;
    const int m2 = std::min(13, 26 / m.sbits);
    if (m2 > m1 && survival_bits(m, m2, m.surv2)) m.sm_m2 = m2;
}

// ---- residency --------------------------------------------------------------
size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

size_t device_bytes(const Machine &m) {
    size_t b = align256(m.memo.size() * 2 + 4) + align256(m.surv.size() * 4 + 4) +
               align256(m.surv2.size() * 4 + 4) + align256(m.tail.size() * 2 + 4);
    if (m.kind == 0) {
        b += align256(m.dtab.size() * 2 + 4) + align256(m.pool.size() * 4);
    } else {
        b += align256(m.off.size() * 4) + align256(m.tgt.size() * 2 + 4) +
             align256(m.pool.size() * 4) + align256(m.band.size() * 4) +
             align256(m.ecl_off.size() * 4) + align256(m.ecl_tgt.size() * 2 + 4) +
             align256(m.l2tab.size() * 2) + align256(m.pool2.size() * 4 + 16) +
             align256(m.memox.size() * 2 + 4);
    }
    return b;
}

// Frees a machine's device image once nothing can still read it: the host
// waits for the machine's last uses on every stream and for its upload, then
// returns the memory to the pool (API calls: evict, unload, new parameters).
void release(pfsm_ctx *ctx, Machine &m) {
    if (!m.dev) return;
    for (auto &u : m.uses) cudaEventSynchronize(u.second);
    if (m.ready) cudaEventSynchronize(m.ready);
    cudaFreeAsync(m.dev, nullptr);
    m.dev = nullptr;
    m.uses.clear();
    ctx->resident_bytes -= m.dev_bytes;
    m.dev_bytes = 0;
}

void drop_host_image(Machine &m) {
    if (m.host_img) cudaFreeHost(m.host_img);
    m.host_img = nullptr;
    m.img_bytes = 0;
}

// Eviction without a host or device synchronisation: stream `s` waits for
// the victim's last use on every stream and for its upload, then frees it
// into the pool at that point of `s`; a later allocation on `s` may reuse
// the memory in stream order.
static void release_async(pfsm_ctx *ctx, Machine &m, cudaStream_t s) {
    if (!m.dev) return;
    for (auto &u : m.uses)
        if (u.first != s) cudaStreamWaitEvent(s, u.second, 0);
    if (m.ready) cudaStreamWaitEvent(s, m.ready, 0);
    cudaFreeAsync(m.dev, s);
    m.dev = nullptr;
    m.uses.clear();
    ctx->resident_bytes -= m.dev_bytes;
    m.dev_bytes = 0;
}

static bool in_use(Machine &m) {
    bool busy = false;
    for (auto &u : m.uses)
        if (cudaEventQuery(u.second) != cudaSuccess) busy = true;
    if (m.ready && cudaEventQuery(m.ready) != cudaSuccess) busy = true;
    cudaGetLastError();   // a pending event is not an error
    return busy;
}

static void forget(pfsm_ctx *ctx, Machine &m) {
    release(ctx, m);
    drop_host_image(m);
    if (m.ready) cudaEventDestroy(m.ready);
    m.ready = nullptr;
}

// Frees the retired machines that nothing reads any more.
void sweep_retired(pfsm_ctx *ctx) {
    for (size_t i = 0; i < ctx->retired.size();) {
        if (in_use(ctx->retired[i])) {
            ++i;
            continue;
        }
        forget(ctx, ctx->retired[i]);
        ctx->retired.erase(ctx->retired.begin() + i);
    }
}

int evict_lru(pfsm_ctx *ctx, uint64_t need, int keep_id, cudaStream_t s) {
    sweep_retired(ctx);
    // retired machines go first, freed in the order of stream `s`
    while (ctx->resident_bytes + need > ctx->budget && !ctx->retired.empty()) {
        Machine &r = ctx->retired.back();
        release_async(ctx, r, s);
        drop_host_image(r);
        if (r.ready) cudaEventDestroy(r.ready);
        ctx->retired.pop_back();
    }
    while (ctx->resident_bytes + need > ctx->budget) {
        Machine *victim = nullptr;
        for (auto &kv : ctx->machines) {
            if (kv.first == keep_id || !kv.second.dev) continue;
            if (kv.second.pin && kv.second.pin == ctx->epoch) continue;
            if (!victim || kv.second.last_use < victim->last_use) victim = &kv.second;
        }
        if (!victim) return PFSM_E_NOMEM;
        release_async(ctx, *victim, s);
        ctx->n_evict++;
    }
    return PFSM_OK;
}

// The device image of `m`, built once in pinned host memory: 256-byte
// aligned sections (prefix table, short-gram table, survival bitmaps, then
// the DFA table or the NFA CSR, records and band image).
static int build_host_image(Machine &m) {
    if (m.host_img) return PFSM_OK;
    const size_t bytes = device_bytes(m);
    void *h = nullptr;
    if (cudaMallocHost(&h, bytes) != cudaSuccess) {
        cudaGetLastError();
        return PFSM_E_NOMEM;
    }
    uint8_t *img = static_cast<uint8_t *>(h);
    memset(img, 0, bytes);
    size_t o = 0;
    auto put = [&](const void *src, size_t n, size_t pad) {
        const size_t at = o;
        if (n) memcpy(img + o, src, n);
        o += align256(n + pad);
        return at;
    };
    m.o_memo = put(m.memo.data(), m.memo.size() * 2, 4);
    m.o_tail = put(m.tail.data(), m.tail.size() * 2, 4);
    m.o_surv = put(m.surv.data(), m.surv.size() * 4, 4);
    m.o_surv2 = put(m.surv2.data(), m.surv2.size() * 4, 4);
    if (m.kind == 0) {
        m.o_tab = put(m.dtab.data(), m.dtab.size() * 2, 4);
        m.o_pool = put(m.pool.data(), m.pool.size() * 4, 0);
    } else {
        m.o_off = put(m.off.data(), m.off.size() * 4, 0);
        m.o_tgt = put(m.tgt.data(), m.tgt.size() * 2, 4);
        m.o_pool = put(m.pool.data(), m.pool.size() * 4, 0);
        m.o_band = put(m.band.data(), m.band.size() * 4, 0);
        m.o_eoff = put(m.ecl_off.data(), m.ecl_off.size() * 4, 0);
        m.o_etgt = put(m.ecl_tgt.data(), m.ecl_tgt.size() * 2, 4);
        m.o_l2tab = put(m.l2tab.data(), m.l2tab.size() * 2, 0);
        // 16 bytes of slack: a record's first words are read together
        m.o_pool2 = put(m.pool2.data(), m.pool2.size() * 4, 16);
        m.o_memox = put(m.memox.data(), m.memox.size() * 2, 4);
    }
    if (o > bytes) {   // layout and size disagree: a bug, fail loudly
        cudaFreeHost(h);
        return PFSM_E_INVAL;
    }
    m.host_img = img;
    m.img_bytes = bytes;
    return PFSM_OK;
}

// The kernels' view of a machine whose image starts at `base`.
static DevMachine dev_view(const Machine &m, uint8_t *base) {
    DevMachine dm{};
    dm.kind = m.kind;
    dm.Q = m.Q;
    dm.S = m.S;
    dm.q0 = m.q0;
    dm.k = m.k;
    dm.sbits = m.sbits;
    dm.memo_n = m.k > 0 ? (1u << (m.k * m.sbits)) : 0;
    dm.Wq = (m.Q + 31) / 32;
    dm.memo = reinterpret_cast<const uint16_t *>(base + m.o_memo);
    dm.tail = m.tail.empty() ? nullptr : reinterpret_cast<const uint16_t *>(base + m.o_tail);
    dm.surv = m.surv.empty() ? nullptr : reinterpret_cast<const uint32_t *>(base + m.o_surv);
    dm.surv_m = m.sm_m;
    dm.surv_words = static_cast<uint32_t>(m.surv.size());
    dm.surv2 = m.surv2.empty() ? nullptr : reinterpret_cast<const uint32_t *>(base + m.o_surv2);
    dm.surv2_m = m.sm_m2;
    if (m.kind == 0) {
        dm.dtab = reinterpret_cast<const uint16_t *>(base + m.o_tab);
        dm.pool = reinterpret_cast<const uint32_t *>(base + m.o_pool);
        dm.pool_n = static_cast<uint32_t>(m.pool.size());
    } else {
        dm.off = reinterpret_cast<const uint32_t *>(base + m.o_off);
        dm.tgt = reinterpret_cast<const uint16_t *>(base + m.o_tgt);
        dm.pool = reinterpret_cast<const uint32_t *>(base + m.o_pool);
        dm.pool_n = static_cast<uint32_t>(m.pool.size());
        dm.band = m.band.empty() ? nullptr : reinterpret_cast<const uint32_t *>(base + m.o_band);
        dm.ecl_off = m.ecl_off.empty() ? nullptr : reinterpret_cast<const uint32_t *>(base + m.o_eoff);
        dm.ecl_tgt = m.ecl_off.empty() ? nullptr : reinterpret_cast<const uint16_t *>(base + m.o_etgt);
        dm.l2tab = m.l2tab.empty() ? nullptr : reinterpret_cast<const uint16_t *>(base + m.o_l2tab);
        dm.pool2 = m.l2tab.empty() ? nullptr : reinterpret_cast<const uint32_t *>(base + m.o_pool2);
        dm.memox = m.memox.empty() ? nullptr : reinterpret_cast<const uint16_t *>(base + m.o_memox);
    }
    return dm;
}

// Makes `m` resident for work enqueued on `s`: a resident machine only makes
// `s` wait for its upload (when that has not finished yet); otherwise the
// least recently used machines are evicted in stream order, an image is
// taken from the pool and the pinned host image is copied in on `s`.
int make_resident(pfsm_ctx *ctx, int id, Machine &m, cudaStream_t s) {
    NvtxRange nr("pfsm make_resident");
    m.last_use = ++ctx->clock;
    if (!m.ready && cudaEventCreateWithFlags(&m.ready, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return PFSM_E_CUDA;
    }
    if (m.dev) {
        if (cudaEventQuery(m.ready) != cudaSuccess) {
            cudaGetLastError();
            cudaStreamWaitEvent(s, m.ready, 0);
        }
        return PFSM_OK;
    }
    int st = build_host_image(m);
    if (st) return st;
    const size_t bytes = m.img_bytes;
    st = evict_lru(ctx, bytes, id, s);
    if (st) return st;
    void *p = nullptr;
    if (cudaMallocFromPoolAsync(&p, bytes, ctx->pool, s) != cudaSuccess) {
        cudaGetLastError();
        return PFSM_E_NOMEM;
    }
    if (cudaMemcpyAsync(p, m.host_img, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaEventRecord(m.ready, s) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeAsync(p, s);
        return PFSM_E_CUDA;
    }
    m.dev = p;
    m.dev_bytes = bytes;
    m.dm = dev_view(m, static_cast<uint8_t *>(p));
    ctx->resident_bytes += bytes;
    if (m.was_resident) ctx->n_reload++;
    m.was_resident = true;
    return PFSM_OK;
}

// Records that the work just enqueued on `s` reads the images of ms[0..k).
int mark_use(pfsm_ctx *ctx, cudaStream_t s, Machine *const *ms, size_t k) {
    UseRing &r = ctx->use_rings[s];
    cudaEvent_t &ev = r.ev[r.head];
    if (!ev && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return PFSM_E_CUDA;
    }
    r.head = (r.head + 1) % kUseRing;
    if (cudaEventRecord(ev, s) != cudaSuccess) return PFSM_E_CUDA;
    for (size_t i = 0; i < k; ++i) {
        Machine &m = *ms[i];
        bool found = false;
        for (auto &u : m.uses)
            if (u.first == s) {
                u.second = ev;
                found = true;
            }
        if (!found) m.uses.emplace_back(s, ev);
    }
    return PFSM_OK;
}

// Grows a device scratch buffer to at least `need` words (synchronises the
// device when it has to reallocate, which happens once per size class).
int ensure_words(uint32_t **buf, size_t *have, size_t need) {
    if (need <= *have) return PFSM_OK;
    size_t n = std::max(need, 2 * *have);
    if (*buf) {
        cudaDeviceSynchronize();
        cudaFree(*buf);
        *buf = nullptr;
        *have = 0;
    }
    if (cudaMalloc(buf, n * 4) != cudaSuccess) {
        cudaGetLastError();
        *buf = nullptr;
        return PFSM_E_NOMEM;
    }
    *have = n;
    return PFSM_OK;
}

Slot *get_slot(pfsm_ctx *ctx, cudaStream_t s) {
    std::lock_guard<std::mutex> g(ctx->mu);
    auto it = ctx->slots.find(s);
    if (it != ctx->slots.end()) return &it->second;
    Slot sl;
    void *p = nullptr;
    const size_t bytes = 64 + static_cast<size_t>(kCarryCap) * 16;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    sl.status = static_cast<unsigned long long *>(p);
    sl.carry_n = reinterpret_cast<uint32_t *>(static_cast<uint8_t *>(p) + 16);
    sl.carry = reinterpret_cast<uint32_t *>(static_cast<uint8_t *>(p) + 64);
    if (cudaMallocHost(&sl.host_status, 2 * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(p);
        return nullptr;
    }
    for (int i = 0; i < 2 * kEventRing; ++i) cudaEventCreate(&sl.ev[i]);
    return &ctx->slots.emplace(s, sl).first->second;
}

void fill_defaults(const Machine &m, pfsm_params &p) {
    if (p.prefix_k == 0) p.prefix_k = default_k(m);
    // tile 0 = automatic: 16 KiB, smaller for texts too short to fill the GPU
    if (p.halo == 0) p.halo = 2048;
    // threads 0 = automatic: 512, fewer for texts too short to fill the GPU

    if (p.table_smem == 0) p.table_smem = -1;
    // settling cap: 8 steps past the prefix (3 past a second-level record)
    // hands the few long-lived instances to the exact path early
    if (p.settle == 0) p.settle = 8;
    if (p.partition == 0) p.partition = m.kind == 0 ? 2 : 1;
}

int validate_params(const Machine &m, const pfsm_params &p) {
    if (p.prefix_k < -1 || p.prefix_k > 8) return PFSM_E_INVAL;
    if (p.prefix_k > 0 && p.prefix_k * m.sbits > 16) return PFSM_E_INVAL;
    if (p.tile != 0 && (p.tile < 4096 || p.tile > 49152 || p.tile % 4096)) return PFSM_E_INVAL;
    if (p.halo < 16 || p.halo > 16384 || p.halo % 16) return PFSM_E_INVAL;
    if (p.threads != 0 && p.threads != 128 && p.threads != 256 && p.threads != 512)
        return PFSM_E_INVAL;
    if (p.spt != 0 && p.spt != 8 && p.spt != 32) return PFSM_E_INVAL;
    if (p.table_smem < -1 || p.table_smem > 1) return PFSM_E_INVAL;
    if (p.ctas_per_sm < 0 || p.ctas_per_sm > 8) return PFSM_E_INVAL;
    if (p.settle < -1 || p.settle > 63) return PFSM_E_INVAL;
    if (p.partition < 0 || p.partition > 2) return PFSM_E_INVAL;
    if (!m.ecl_off.empty() && p.prefix_k == -1) return PFSM_E_INVAL;   // see finish_load
    return PFSM_OK;
}

// Apply the params' prefix depth to the machine (rebuilding its table). An
// NFA whose records do not fit 16-bit pool offsets at that depth gets a
// smaller one when `may_lower` (the depth was the default); otherwise the
// previous table is rebuilt and E_INVAL returned.
int apply_k(pfsm_ctx *ctx, Machine &m, bool may_lower) {
    const int k = m.params.prefix_k < 0 ? 0 : m.params.prefix_k;
    if (k == m.k && (k == 0 || !m.memo.empty())) return PFSM_OK;
    const int old_k = m.k;
    // a machine with epsilon edges keeps k >= 1: no start steps from a bare q0
    const int floor_k = m.ecl_off.empty() ? 0 : 1;
    release(ctx, m);
    drop_host_image(m);   // the prefix tables change: rebuild the image
    m.k = std::max(k, floor_k);
    while (!build_memo(m)) {
        if (!may_lower || m.k - 1 < floor_k) {
            m.k = old_k;
            build_memo(m);
            m.params.prefix_k = old_k > 0 ? old_k : -1;
            return PFSM_E_INVAL;
        }
        --m.k;   // k = 0 always builds (no table)
    }
    m.params.prefix_k = m.k > 0 ? m.k : -1;
    return PFSM_OK;
}

struct Plan {
    ScanArgs a;
    int threads, grid;
    uint32_t smem;
};

// Launch geometry and shared-memory layout of one scan.
int plan_scan(pfsm_ctx *ctx, const Machine &m, const uint8_t *text, uint64_t n, Plan &pl) {
    const pfsm_params &p = m.params;
    ScanArgs &a = pl.a;
    memset(&a, 0, sizeof(a));
    a.text = text;
    a.n = static_cast<uint32_t>(n);
    // starts per thread per filter round: 32 for long texts; 8 for texts too
    // short to give every SM 16 warps of 32-start threads (four times the
    // warps, so more latency is hidden)
    int spt = p.spt;
    if (spt == 0) spt = n < 16ull * ctx->nsm * 32 * FILTER_SPT ? 8 : FILTER_SPT;
    a.spt = spt;
    int threads = p.threads;
    if (threads == 0) {
        // keep at least two filter rounds' worth of tiles per SM
        threads = 512;
        while (threads > 128 && n < 2ull * ctx->nsm * static_cast<uint64_t>(spt) * threads)
            threads /= 2;
    }
    // the NFA kernel with a producer warp runs 15 filtering warps: 16 warps
    // in all put four on each of an SM's sub-partitions, whose registers then
    // allow 128 per thread (a seventeenth warp would cut that to 96 and spill)
    if (m.kind == 1 && spt == FILTER_SPT && threads == 512) threads = 480;
    uint32_t tile = static_cast<uint32_t>(p.tile);
    if (tile == 0 && spt == 8) {
        tile = static_cast<uint32_t>(spt) * threads;   // one filter round: the most CTAs
    } else if (tile == 0) {
        // at least two tiles per SM when the text allows it
        const uint64_t want = n / (2ull * ctx->nsm);
        tile = static_cast<uint32_t>(std::min<uint64_t>(16384, std::max<uint64_t>(4096, (want + 4095) & ~4095ull)));
        // whole filter rounds
        const uint32_t round = static_cast<uint32_t>(spt) * threads;
        tile = std::max<uint32_t>(round, tile / round * round);
    }
    a.tile = tile;
    a.halo = p.halo;
    a.ntiles = static_cast<uint32_t>((n + tile - 1) / tile);
    a.text_buf = (tile + p.halo + 32 + 127) & ~127u;
    // staged tiles: one in use, one being prepared, one in flight; a short
    // text gives a CTA one or two tiles, and two buffers leave more shared
    // memory for CTAs
    a.nbuf = spt == 8 ? 2 : 3;
    a.shift = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(text) & 15);
    a.Q = m.Q;
    a.S = m.S;
    a.q0 = m.q0;
    a.k = m.k;
    a.sbits = m.sbits;
    a.memo_n = m.dm.memo_n;
    a.memo = m.dm.memo;
    a.tail = m.dm.tail;
    a.ecl_off = m.dm.ecl_off;
    a.ecl_tgt = m.dm.ecl_tgt;
    a.dtab = m.dm.dtab;
    a.off = m.dm.off;
    a.tgt = m.dm.tgt;
    a.pool = m.dm.pool;
    a.l2tab = m.dm.l2tab;
    a.memox = m.dm.memox;
    a.pool2 = m.dm.pool2;
    a.pool_n = m.dm.pool_n;
    a.band = m.dm.band;
    a.surv = m.dm.surv;
    a.surv_m = m.dm.surv_m;
    a.surv_words = m.dm.surv_words;
    a.surv2 = m.dm.surv2;
    a.surv2_m = m.dm.surv2_m;
    a.Wq = m.kind == 1 ? m.dm.Wq : 0;
    uint32_t tab_bytes = m.kind == 0 ? ((static_cast<uint32_t>(m.Q) * m.S + 1) / 2) * 4 : 0;
    // table placement: shared memory when asked, or (auto) when small
    a.tab_smem = 0;
    if (m.kind == 0) {
        if (p.table_smem == 1) a.tab_smem = 1;
        else if (p.table_smem == -1 && tab_bytes <= 48 * 1024) a.tab_smem = 1;
    }
    const int kmask = m.kind == 0 ? 1 : 2;
    a.stage_n = m.kind == 0 ? STAGE : 32;
    SmemNeed need{};
    // with a deep filter few starts reach the prefix table: leave it in
    // global memory and keep shared memory for occupancy
    const bool deep = !m.surv2.empty();
    need.memo_bytes = deep ? 0u : static_cast<uint32_t>(((m.memo.size() + 1) / 2) * 4 + 4);
    if (m.memo.empty()) need.memo_bytes = 0;
    need.tab_bytes = a.tab_smem ? tab_bytes : 0;
    need.band_bytes = m.kind == 1 ? static_cast<uint32_t>(m.band.size() * 4) : 0;
    // the NFA records are read by every start that reaches settling: shared
    // memory when they fit
    need.pool_bytes = ((m.kind == 1 && m.pool.size() * 4 <= 64 * 1024) ||
                       (m.kind == 0 && m.pool.size() > 1 && m.pool.size() * 4 <= 16 * 1024))
                          ? static_cast<uint32_t>(m.pool.size() * 4) : 0;
    a.settle_steps = m.params.settle > 0 ? m.params.settle : 0;
    need.surv_bytes = static_cast<uint32_t>(m.surv.size() * 4);
    // 2-grams of bytes: the shallow bitmap as one byte per 2-gram (64 KB),
    // so that the gram index is the load offset
    const bool byte_table = m.sbits == 8 && m.sm_m == 2 && !m.surv.empty();
    if (byte_table) need.surv_bytes = 1u << 16;
    // warp-wide bitsets of sets too large for a lane: shared memory keeps
    // their atomics on chip
    need.coop_bytes = m.kind == 1 ? static_cast<uint32_t>((threads / 32) * 2 * m.dm.Wq * 4) : 0u;
    uint32_t smem = 0;
    bool fit = false;
    for (int attempt = 0; attempt < 8 && !fit; ++attempt) {
        a.surv_bytes = byte_table && need.surv_bytes == (1u << 16);
        smem = layout_smem(a, kmask, threads, need);
        if (smem <= kSmemMax - kSmemStatic) { fit = true; break; }
        // shrink, cheapest loss first: match staging, then table copies
        // (largest first)
        if (a.stage_n > 32) a.stage_n = 32;
        else if (need.surv_bytes > (1u << 15) && byte_table) need.surv_bytes = static_cast<uint32_t>(m.surv.size() * 4);
        else if (need.coop_bytes) need.coop_bytes = 0;   // rare: sets of more than 8 states
        else if (need.pool_bytes) need.pool_bytes = 0;
        else if (need.memo_bytes) need.memo_bytes = 0;
        else if (need.band_bytes) need.band_bytes = 0;
        else if (need.tab_bytes && p.table_smem == -1) { need.tab_bytes = 0; a.tab_smem = 0; }
        else break;
    }
    if (!fit) return PFSM_E_INVAL;
    int occ = max_ctas_per_sm(m.kind, m.sbits, threads, smem, a.tab_smem != 0, spt);
    if (occ <= 0) return PFSM_E_INVAL;
    if (p.ctas_per_sm > 0) occ = std::min(occ, p.ctas_per_sm);
    pl.threads = threads;
    pl.smem = smem;
    pl.grid = static_cast<int>(std::min<uint64_t>(a.ntiles, static_cast<uint64_t>(ctx->nsm) * occ));
    if (pl.grid < 1) pl.grid = 1;
    return PFSM_OK;
}

// Accumulate the durations of timed launches, oldest first; `keep` pairs
// may stay pending (0 drains all of them, waiting for their completion).
void collect_timing(pfsm_ctx *ctx, Slot *slot, int keep) {
    while (slot->ev_pending > keep) {
        const int i = (slot->ev_head - slot->ev_pending + kEventRing) % kEventRing;
        float ms = 0.f;
        cudaEventSynchronize(slot->ev[2 * i + 1]);
        if (cudaEventElapsedTime(&ms, slot->ev[2 * i], slot->ev[2 * i + 1]) == cudaSuccess) {
            ctx->time_ms += ms;
            ctx->time_launches += 1;
        }
        slot->ev_pending--;
    }
}

int scan_enqueue(pfsm_ctx *ctx, pfsm_aut aut, const uint8_t *text, uint64_t n, uint32_t *out,
                 uint64_t cap, unsigned long long *status, Slot *slot, cudaStream_t s) {
    NvtxRange nr("pfsm scan (plan, tile kernel, carry)");
    auto it = ctx->machines.find(aut);
    if (it == ctx->machines.end()) return PFSM_E_NOENT;
    Machine &m = it->second;
    int st = make_resident(ctx, aut, m, s);
    if (st) return st;
    if (cudaMemsetAsync(status, 0, 2 * sizeof(unsigned long long), s) != cudaSuccess)
        return PFSM_E_CUDA;
    if (n == 0) return PFSM_OK;
    Plan pl;
    st = plan_scan(ctx, m, text, n, pl);
    if (st) return st;
    pl.a.out = out;
    pl.a.cap = cap;
    pl.a.status = status;
    pl.a.hold_tiles = ctx->hold_tiles ? 1u : 0u;
    pl.a.carry = slot->carry;
    pl.a.carry_n = slot->carry_n;
    // lazy partitioning: no carry queue, instances continue in place.
    // Chained: the slot's carry buffer holds kCarryCap DFA entries of 4
    // words, or for an NFA kCarryCap / 4 entries of 8 words followed by a
    // pool of 2 kCarryCap states for the larger sets
    pl.a.carry_cap = m.params.partition == 1 ? 0u : m.kind == 0 ? kCarryCap : kCarryCap / 4;
    pl.a.cpool = m.kind == 1 ? reinterpret_cast<uint16_t *>(slot->carry + 2 * kCarryCap) : nullptr;
    pl.a.cpool_cap = m.kind == 1 ? 2 * kCarryCap : 0u;
    if (pl.a.carry_cap && ctx->test_carry_cap) pl.a.carry_cap = std::min(pl.a.carry_cap, ctx->test_carry_cap);
    if (pl.a.cpool_cap && ctx->test_cpool_cap) pl.a.cpool_cap = std::min(pl.a.cpool_cap, ctx->test_cpool_cap);
    if (m.kind == 1 && !pl.a.coop_smem) {
        // one pair of bitsets per warp of the tile kernel and, when the scan
        // is chained, of the carry kernel (nsm CTAs of up to 256 threads)
        size_t warps = static_cast<size_t>(pl.grid) * (pl.threads / 32);
        if (pl.a.carry_cap)
            warps = std::max(warps, static_cast<size_t>(ctx->nsm) * (std::min(pl.threads, 256) / 32));
        const size_t need = warps * 2 * m.dm.Wq;
        if (ensure_words(&slot->coop, &slot->coop_words, need)) return PFSM_E_NOMEM;
        pl.a.coop_g = slot->coop;
    }
    if (pl.a.carry_cap && cudaMemsetAsync(slot->carry_n, 0, 8 * sizeof(uint32_t), s) != cudaSuccess)
        return PFSM_E_CUDA;
    int ev = -1;
    if (ctx->timing) {
        collect_timing(ctx, slot, kEventRing - 1);
        ev = slot->ev_head;
        cudaEventRecord(slot->ev[2 * ev], s);
    }
    cudaError_t e = launch_scan(pl.a, m.kind, pl.threads, pl.grid, pl.smem, s);
    if (ev >= 0) {
        cudaEventRecord(slot->ev[2 * ev + 1], s);
        slot->ev_head = (slot->ev_head + 1) % kEventRing;
        slot->ev_pending++;
    }
    if (e != cudaSuccess) return PFSM_E_CUDA;
    if (m.kind == 0 && pl.a.carry_cap > 0) {
        NvtxRange nr("pfsm carry_dfa launch");
        e = launch_carry(pl.a, 2 * ctx->nsm, s);
        if (e != cudaSuccess) return PFSM_E_CUDA;
    } else if (m.kind == 1 && pl.a.carry_cap > 0) {
        NvtxRange nr("pfsm carry_nfa launch");
        e = launch_carry_nfa(pl.a, ctx->nsm, std::min(pl.threads, 256), s);
        if (e != cudaSuccess) return PFSM_E_CUDA;
    }
    {
        Machine *mp = &m;
        st = mark_use(ctx, s, &mp, 1);
        if (st) return st;
    }
    return PFSM_OK;
}

int finish_status(const unsigned long long *hs, uint64_t cap, uint64_t *n_matches) {
    if (n_matches) *n_matches = hs[0];
    if (hs[1] & ERR_CHECK) return PFSM_E_CHECK;
    if (hs[1] & ERR_TIMEOUT) return PFSM_E_TIMEOUT;
    if (hs[1] & ERR_SYMBOL) return PFSM_E_INVAL;
    if (hs[0] > cap) return PFSM_E_OVERFLOW;
    return PFSM_OK;
}

}  // namespace pfsm

// =========================================================================
extern "C" {

int pfsm_ctx_create(int device, uint64_t budget_bytes, pfsm_ctx **out) {
    if (!out) return PFSM_E_INVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return PFSM_E_CUDA;
    }
    if (device < 0 || device >= ndev) return PFSM_E_INVAL;
    DeviceGuard g(device);
    pfsm_ctx *c = new pfsm_ctx();
    c->device = device;
    c->budget = budget_bytes ? budget_bytes : kDefaultBudget;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        delete c;
        return PFSM_E_CUDA;
    }
    c->nsm = prop.multiProcessorCount;
    c->smem_sm = static_cast<uint32_t>(prop.sharedMemPerMultiprocessor);
    c->smem_rsv = static_cast<uint32_t>(prop.reservedSharedMemPerBlock);
    // machine images come from a pool of this context that keeps freed
    // memory for reuse (evictions and reloads cost no allocator round trip)
    cudaMemPoolProps pp;
    memset(&pp, 0, sizeof(pp));
    pp.allocType = cudaMemAllocationTypePinned;
    pp.location.type = cudaMemLocationTypeDevice;
    pp.location.id = device;
    if (cudaMemPoolCreate(&c->pool, &pp) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return PFSM_E_CUDA;
    }
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    *out = c;
    return PFSM_OK;
}

int pfsm_ctx_destroy(pfsm_ctx *ctx) {
    if (!ctx) return PFSM_OK;
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    for (auto &kv : ctx->machines) forget(ctx, kv.second);
    for (auto &m : ctx->retired) forget(ctx, m);
    ctx->retired.clear();
    for (auto &kv : ctx->use_rings)
        for (int i = 0; i < kUseRing; ++i)
            if (kv.second.ev[i]) cudaEventDestroy(kv.second.ev[i]);
    for (auto &kv : ctx->slots) {
        cudaFree(kv.second.coop);
        cudaFree(kv.second.status);
        cudaFreeHost(kv.second.host_status);
        for (int i = 0; i < 2 * kEventRing; ++i) cudaEventDestroy(kv.second.ev[i]);
    }
    batch_free(ctx);
    cudaDeviceSynchronize();
    if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
    delete ctx;
    return PFSM_OK;
}

static int finish_load(pfsm_ctx *ctx, Machine &&m, pfsm_aut *out_id) {
    NvtxRange nr("pfsm load (tables, survival bitmaps, upload)");
    m.sbits = ceil_log2(m.S);
    fill_defaults(m, m.params);
    m.k = m.params.prefix_k < 0 ? 0 : m.params.prefix_k;
    if (m.k * m.sbits > 16) m.k = 16 / m.sbits;
    if (!m.ecl_off.empty() && m.k < 1) m.k = 1;   // epsilon edges: no start steps from a bare q0
    while (!build_memo(m)) {
        if (--m.k <= 0) {
            if (!m.ecl_off.empty()) return PFSM_E_INVAL;
            m.k = 0;
            build_memo(m);
            break;
        }
    }
    m.params.prefix_k = m.k > 0 ? m.k : -1;
    build_survival(m);
    DeviceGuard g(ctx->device);
    const int id = ctx->next_id++;
    auto &slot = ctx->machines[id];
    slot = std::move(m);
    ctx->n_loads++;
    int st = make_resident(ctx, id, slot, nullptr);
    if (!st && cudaEventSynchronize(slot.ready) != cudaSuccess) st = PFSM_E_CUDA;
    if (st) {
        drop_host_image(slot);
        if (slot.ready) cudaEventDestroy(slot.ready);
        ctx->machines.erase(id);
        return st;
    }
    *out_id = id;
    return PFSM_OK;
}

int pfsm_load_dfa(pfsm_ctx *ctx, const int16_t *delta, int32_t Q, int32_t S, int32_t q0,
                  int32_t dead, const uint8_t *is_final, pfsm_aut *out_id) {
    if (!ctx || !delta || !is_final || !out_id) return PFSM_E_INVAL;
    if (Q < 1 || Q > 32767 || S < 1 || S > 256) return PFSM_E_INVAL;
    if (q0 < 0 || q0 >= Q || dead < -1 || dead >= Q) return PFSM_E_INVAL;
    if (dead == q0) return PFSM_E_INVAL;
    for (size_t i = 0; i < (size_t)Q * S; ++i)
        if (delta[i] < 0 || delta[i] >= Q) return PFSM_E_INVAL;
    if (dead >= 0) {
        if (is_final[dead]) return PFSM_E_INVAL;
        for (int a = 0; a < S; ++a)
            if (delta[(size_t)dead * S + a] != dead) return PFSM_E_INVAL;
    }
    Machine m;
    m.kind = 0;
    m.Q = Q;
    m.S = S;
    m.q0 = q0;
    m.dead = dead;
    m.fin.assign(is_final, is_final + Q);
    m.dtab.resize((size_t)Q * S + ((size_t)Q * S & 1));
    for (size_t i = 0; i < (size_t)Q * S; ++i) {
        const int t = delta[i];
        m.dtab[i] = t == dead ? DEAD16
                              : static_cast<uint16_t>(t | (is_final[t] ? FINAL_BIT : 0));
    }
    return finish_load(ctx, std::move(m), out_id);
}

static int load_nfa(pfsm_ctx *ctx, const uint32_t *delta_bits, const uint32_t *eps_bits,
                    int32_t Q, int32_t S, int32_t q0, const uint8_t *is_final, pfsm_aut *out_id) {
    if (!ctx || !delta_bits || !is_final || !out_id) return PFSM_E_INVAL;
    if (Q < 1 || Q > 32767 || S < 1 || S > 256) return PFSM_E_INVAL;
    if (q0 < 0 || q0 >= Q) return PFSM_E_INVAL;
    const int W = (Q + 31) / 32;
    const uint32_t lastmask = (Q % 32) ? ((1u << (Q % 32)) - 1) : 0xFFFFFFFFu;
    Machine m;
    m.kind = 1;
    m.Q = Q;
    m.S = S;
    m.q0 = q0;
    m.fin.assign(is_final, is_final + Q);
    m.off.resize((size_t)Q * S + 1);
    uint64_t e = 0;
    for (size_t r = 0; r < (size_t)Q * S; ++r) {
        m.off[r] = static_cast<uint32_t>(e);
        const uint32_t *row = delta_bits + r * W;
        if (row[W - 1] & ~lastmask) return PFSM_E_INVAL;   // a target >= Q
        for (int w = 0; w < W; ++w) {
            uint32_t x = row[w];
            while (x) {
                const int b = __builtin_ctz(x);
                x &= x - 1;
                const int t = w * 32 + b;
                m.tgt.push_back(static_cast<uint16_t>(t | (is_final[t] ? FINAL_BIT : 0)));
                ++e;
            }
        }
        if (e > 0xFFFFFFFFull) return PFSM_E_INVAL;
    }
    m.off[(size_t)Q * S] = static_cast<uint32_t>(e);
    // epsilon edges kept for run time: the states each state reaches through
    // them (breadth first; the state itself excluded)
    bool has_eps = false;
    if (eps_bits) {
        for (size_t x = 0; x < (size_t)Q * W; ++x) has_eps |= eps_bits[x] != 0;
        if (eps_bits[(size_t)(Q - 1) * W + W - 1] & ~lastmask) return PFSM_E_INVAL;
        for (int q = 0; q < Q && has_eps; ++q)
            if (eps_bits[(size_t)q * W + W - 1] & ~lastmask) return PFSM_E_INVAL;
    }
    if (has_eps) {
        m.ecl_off.assign(static_cast<size_t>(Q) + 1, 0);
        std::vector<int> seen(Q, -1), queue;
        for (int q = 0; q < Q; ++q) {
            m.ecl_off[q] = static_cast<uint32_t>(m.ecl_tgt.size());
            queue.assign(1, q);
            seen[q] = q;
            std::vector<uint16_t> reach;
            for (size_t h = 0; h < queue.size(); ++h) {
                const uint32_t *row = eps_bits + (size_t)queue[h] * W;
                for (int w = 0; w < W; ++w) {
                    uint32_t x = row[w];
                    while (x) {
                        const int t = w * 32 + __builtin_ctz(x);
                        x &= x - 1;
                        if (seen[t] == q) continue;
                        seen[t] = q;
                        queue.push_back(t);
                        reach.push_back(static_cast<uint16_t>(t | (is_final[t] ? FINAL_BIT : 0)));
                    }
                }
            }
            std::sort(reach.begin(), reach.end());
            m.ecl_tgt.insert(m.ecl_tgt.end(), reach.begin(), reach.end());
        }
        m.ecl_off[Q] = static_cast<uint32_t>(m.ecl_tgt.size());
        if (m.ecl_tgt.empty()) m.ecl_tgt.push_back(0);
    }
    // band rows: delta(q, a) inside q+1..q+8 for every symbol (alphabets of
    // at most 4 symbols), with the finality of each target beside it; a
    // machine with epsilon edges reads the CSR rows and their closures
    if (S <= 4 && !has_eps) {
        m.band.assign(static_cast<size_t>(Q) + W, 0u);
        for (int q = 0; q < Q; ++q) {
            uint32_t row = 0;
            bool fits = true;
            for (int a = 0; a < S && fits; ++a) {
                for (uint32_t x = m.off[(size_t)q * S + a]; x < m.off[(size_t)q * S + a + 1]; ++x) {
                    const int t = m.tgt[x] & 0x7FFF;
                    const int d = t - q - 1;
                    if (d < 0 || d > 7) {
                        fits = false;
                        break;
                    }
                    row |= 1u << (8 * a + d);
                }
            }
            m.band[q] = (fits && row != BAND_CSR) ? row : BAND_CSR;
        }
        for (int q = 0; q < Q; ++q)
            if (is_final[q]) m.band[Q + (q >> 5)] |= 1u << (q & 31);
    }
    if (m.tgt.empty()) m.tgt.push_back(0);
    return finish_load(ctx, std::move(m), out_id);
}

int pfsm_load_nfa(pfsm_ctx *ctx, const uint32_t *delta_bits, int32_t Q, int32_t S, int32_t q0,
                  const uint8_t *is_final, pfsm_aut *out_id) {
    return load_nfa(ctx, delta_bits, nullptr, Q, S, q0, is_final, out_id);
}

int pfsm_load_nfa_eps(pfsm_ctx *ctx, const uint32_t *delta_bits, const uint32_t *eps_bits,
                      int32_t Q, int32_t S, int32_t q0, const uint8_t *is_final,
                      pfsm_aut *out_id) {
    if (!eps_bits) return PFSM_E_INVAL;
    return load_nfa(ctx, delta_bits, eps_bits, Q, S, q0, is_final, out_id);
}

int pfsm_evict(pfsm_ctx *ctx, pfsm_aut aut) {
    NvtxRange nr("pfsm evict");
    if (!ctx) return PFSM_E_INVAL;
    auto it = ctx->machines.find(aut);
    if (it == ctx->machines.end()) return PFSM_E_NOENT;
    DeviceGuard g(ctx->device);
    if (it->second.dev) {
        release(ctx, it->second);
        ctx->n_evict++;
    }
    return PFSM_OK;
}

int pfsm_aut_bytes(pfsm_ctx *ctx, pfsm_aut aut, uint64_t *bytes, int32_t *resident) {
    if (!ctx) return PFSM_E_INVAL;
    auto it = ctx->machines.find(aut);
    if (it == ctx->machines.end()) return PFSM_E_NOENT;
    if (bytes) *bytes = device_bytes(it->second);
    if (resident) *resident = it->second.dev ? 1 : 0;
    return PFSM_OK;
}

int pfsm_unload(pfsm_ctx *ctx, pfsm_aut aut) {
    if (!ctx) return PFSM_E_INVAL;
    auto it = ctx->machines.find(aut);
    if (it == ctx->machines.end()) return PFSM_E_NOENT;
    DeviceGuard g(ctx->device);
    Machine m = std::move(it->second);
    ctx->machines.erase(it);
    // scans in flight may still read the image: retire it instead of waiting
    if (m.dev && in_use(m)) ctx->retired.push_back(std::move(m));
    else forget(ctx, m);
    sweep_retired(ctx);
    return PFSM_OK;
}

int pfsm_set_params(pfsm_ctx *ctx, pfsm_aut aut, const pfsm_params *p) {
    if (!ctx) return PFSM_E_INVAL;
    auto it = ctx->machines.find(aut);
    if (it == ctx->machines.end()) return PFSM_E_NOENT;
    Machine &m = it->second;
    pfsm_params np{};
    if (p) np = *p;
    const bool default_depth = np.prefix_k == 0;
    fill_defaults(m, np);
    int st = validate_params(m, np);
    if (st) return st;
    DeviceGuard g(ctx->device);
    m.params = np;
    return apply_k(ctx, m, default_depth);
}

int pfsm_get_params(pfsm_ctx *ctx, pfsm_aut aut, pfsm_params *out) {
    if (!ctx || !out) return PFSM_E_INVAL;
    auto it = ctx->machines.find(aut);
    if (it == ctx->machines.end()) return PFSM_E_NOENT;
    *out = it->second.params;
    return PFSM_OK;
}

int pfsm_scan_async(pfsm_ctx *ctx, pfsm_aut aut, const uint8_t *text_dev, uint64_t n,
                    pfsm_match *out_dev, uint64_t cap, uint64_t *status_dev, void *stream) {
    if (!ctx || !status_dev) return PFSM_E_INVAL;
    if (n >= (1ull << 32)) return PFSM_E_INVAL;
    if ((n > 0 && !text_dev) || (cap > 0 && !out_dev)) return PFSM_E_INVAL;
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Slot *slot = get_slot(ctx, s);
    if (!slot) return PFSM_E_NOMEM;
    return scan_enqueue(ctx, aut, text_dev, n, reinterpret_cast<uint32_t *>(out_dev), cap,
                        reinterpret_cast<unsigned long long *>(status_dev), slot, s);
}

int pfsm_scan(pfsm_ctx *ctx, pfsm_aut aut, const uint8_t *text_dev, uint64_t n,
              pfsm_match *out_dev, uint64_t cap, uint64_t *n_matches, void *stream) {
    if (!ctx || !n_matches) return PFSM_E_INVAL;
    if (n >= (1ull << 32)) return PFSM_E_INVAL;
    if ((n > 0 && !text_dev) || (cap > 0 && !out_dev)) return PFSM_E_INVAL;
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Slot *slot = get_slot(ctx, s);
    if (!slot) return PFSM_E_NOMEM;
    int st = scan_enqueue(ctx, aut, text_dev, n, reinterpret_cast<uint32_t *>(out_dev), cap,
                          slot->status, slot, s);
    if (st) return st;
    if (cudaMemcpyAsync(slot->host_status, slot->status, 2 * sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return PFSM_E_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return PFSM_E_CUDA;
    return finish_status(slot->host_status, cap, n_matches);
}

int pfsm_get_stats(pfsm_ctx *ctx, pfsm_stats *out) {
    if (!ctx || !out) return PFSM_E_INVAL;
    {
        DeviceGuard g(ctx->device);
        sweep_retired(ctx);   // unloaded images whose scans have completed
    }
    out->resident_bytes = ctx->resident_bytes;
    out->budget_bytes = ctx->budget;
    out->loads = ctx->n_loads;
    out->evictions = ctx->n_evict;
    out->reloads = ctx->n_reload;
    int r = 0;
    for (auto &kv : ctx->machines) r += kv.second.dev != nullptr;
    out->resident = r;
    out->loaded = static_cast<int32_t>(ctx->machines.size());
    return PFSM_OK;
}

int pfsm_set_timing(pfsm_ctx *ctx, int enable) {
    if (!ctx) return PFSM_E_INVAL;
    DeviceGuard g(ctx->device);
    for (auto &kv : ctx->slots) kv.second.ev_pending = 0;
    ctx->timing = enable != 0;
    ctx->time_ms = 0.0;
    ctx->time_launches = 0;
    return PFSM_OK;
}

int pfsm_test_hold_tiles(pfsm_ctx *ctx, int32_t enable) {
    if (!ctx) return PFSM_E_INVAL;
    ctx->hold_tiles = enable != 0;
    return PFSM_OK;
}

int pfsm_test_carry_cap(pfsm_ctx *ctx, uint32_t entries, uint32_t pool_states) {
    if (!ctx) return PFSM_E_INVAL;
    ctx->test_carry_cap = entries;
    ctx->test_cpool_cap = pool_states;
    return PFSM_OK;
}

int pfsm_kernel_time(pfsm_ctx *ctx, double *ms, uint64_t *launches) {
    if (!ctx) return PFSM_E_INVAL;
    DeviceGuard g(ctx->device);
    for (auto &kv : ctx->slots) collect_timing(ctx, &kv.second, 0);
    if (ms) *ms = ctx->time_ms;
    if (launches) *launches = ctx->time_launches;
    return PFSM_OK;
}

const char *pfsm_strerror(int status) {
    switch (status) {
        case PFSM_OK: return "ok";
        case PFSM_E_INVAL: return "invalid argument, table or text symbol";
        case PFSM_E_NOMEM: return "out of device memory or residency budget";
        case PFSM_E_OVERFLOW: return "more matches than the output capacity";
        case PFSM_E_NOENT: return "unknown automaton id";
        case PFSM_E_TIMEOUT: return "a bounded device wait expired";
        case PFSM_E_CUDA: return "CUDA runtime error";
        case PFSM_E_CHECK: return "a device bounds check failed (checked build)";
        default: return "unknown status";
    }
}

}  // extern "C"
