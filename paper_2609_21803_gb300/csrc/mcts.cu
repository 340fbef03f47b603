// mcts.cu -- Monte Carlo tree search over mode orders (the comparison policy
// of Sec. IV-A / IV-B): a host-side UCT tree whose pools of orders are solved
// by the GPU evaluator.  The readings of the tree (slots, selection,
// expansion, rollout, virtual loss, exhaustion, reward timing, draws) are
// stated in comet_mcts.h.
//
// Host code only: the search makes no CUDA call; comet_plan_mcts reaches
// the GPU through comet_eval_modes and comet_plan.

#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <chrono>
#include <limits>
#include <new>
#include <unordered_map>
#include <vector>

#include "comet.h"
#include "comet_internal.h"
#include "comet_mcts.h"
#include "problem_internal.h"

namespace {

comet_status mfail(comet_status st, const char* msg) {
    comet::set_error(msg);
    return st;
}

constexpr int kPushFree = 12;
constexpr double kInf = std::numeric_limits<double>::infinity();

uint64_t splitmix64(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// pushing grammar: a contact follows a contact only on an adjacent face of
// the cyclic face list; no mode repeats; free motion joins anything
bool push_ok(int a, int b) {
    if (a == b) return false;
    if (a == kPushFree || b == kPushFree) return true;
    const int d = ((a / 3 - b / 3) % 4 + 4) % 4;
    return d == 1 || d == 3;
}

struct Node {
    uint16_t prefix[COMET_MAX_SEGMENTS];
    int32_t len;
    bool stop, exhausted;
    int64_t n;
    double w;
    std::vector<int32_t> untried;                      // slots, ascending
    std::vector<std::pair<int32_t, int32_t>> children;  // (slot, node), ascending slot
};

}  // namespace

static_assert(sizeof(comet_mcts_opts) == 64, "comet_mcts_opts layout");
static_assert(sizeof(comet_mcts_stats) == 40, "comet_mcts_stats layout");

struct comet_mcts {
    comet_mcts_opts o;
    std::vector<int> alpha;
    std::vector<Node> nodes;
    uint64_t ctr = 0;
    double best = kInf;
    int64_t issued = 0;
    std::unordered_map<uint64_t, std::pair<double, double>> results;  // code -> (cost, viol)
    std::vector<uint64_t> result_codes;
    // the pool being filled / waiting for tell: orders and, per code, paths
    std::vector<std::vector<uint16_t>> pool;
    std::vector<uint64_t> pool_codes;
    std::unordered_map<uint64_t, std::vector<std::vector<int32_t>>> waiting;
    bool asked = false;

    uint64_t draw() { return splitmix64(o.seed, ctr++); }

    uint64_t code_of(const uint16_t* m, int len) const {
        const uint64_t base = (uint64_t)o.n_modes + 1;
        uint64_t code = (uint64_t)len, p = base;
        for (int i = 0; i < len; ++i) {
            code += ((uint64_t)m[i] + 1) * p;
            p *= base;
        }
        return code;
    }

    // available actions of a prefix, in slot order
    void slots(const uint16_t* prefix, int len, std::vector<int32_t>& out) const {
        out.clear();
        if (len >= 1) out.push_back(0);
        if (len < o.l_max)
            for (int j = 0; j < (int)alpha.size(); ++j) {
                const int m = alpha[j];
                const bool ok = o.grammar == COMET_GRAMMAR_PUSH
                                    ? (len == 0 ? m == kPushFree : push_ok(prefix[len - 1], m))
                                    : true;
                if (ok) out.push_back(1 + j);
            }
    }

    double value(double cost, double viol) const {
        if (!std::isfinite(cost) || !std::isfinite(viol)) return kInf;
        if (o.reward == COMET_MCTS_REWARD_MERIT) return cost + o.merit_mu * std::max(viol - o.eps_feas, 0.0);
        return viol <= o.eps_feas ? cost : kInf;
    }

    double reward(double cost, double viol) const {
        const double v = value(cost, viol);
        if (v == kInf) return 0.0;
        if (v <= 0.0) return 1.0;
        return best / v;
    }

    double merit(double cost, double viol) const {
        const double m = cost + o.merit_mu * std::max(viol - o.eps_feas, 0.0);
        return std::isnan(m) ? kInf : m;
    }

    int32_t new_node(const uint16_t* prefix, int len, bool stop) {
        Node nd;
        memcpy(nd.prefix, prefix, sizeof(uint16_t) * len);
        nd.len = len;
        nd.stop = stop;
        nd.exhausted = stop;
        nd.n = 0;
        nd.w = 0.0;
        if (!stop) slots(prefix, len, nd.untried);
        nodes.push_back(std::move(nd));
        return (int32_t)nodes.size() - 1;
    }

    // one selection -> expansion -> rollout; creates exactly one node
    void attempt() {
        std::vector<int32_t> path;
        int32_t cur = 0;
        path.push_back(cur);
        while (nodes[cur].untried.empty()) {
            const Node& nd = nodes[cur];
            int32_t pick = -1;
            double best_s = -kInf;
            for (const auto& sc : nd.children) {
                const Node& ch = nodes[sc.second];
                if (ch.exhausted) continue;
                const double s = ch.w / (double)ch.n + o.c_uct * std::sqrt(std::log((double)nd.n) / (double)ch.n);
                if (s > best_s) {
                    best_s = s;
                    pick = sc.second;
                }
            }
            if (pick < 0) {  // unreachable while exhaustion is kept up to date
                nodes[cur].exhausted = true;
                return;
            }
            cur = pick;
            path.push_back(cur);
        }
        // expansion
        int32_t slot;
        {
            Node& nd = nodes[cur];
            const size_t i = (size_t)(draw() % (uint64_t)nd.untried.size());
            slot = nd.untried[i];
            nd.untried.erase(nd.untried.begin() + (ptrdiff_t)i);
        }
        uint16_t prefix[COMET_MAX_SEGMENTS];
        int len = nodes[cur].len;
        memcpy(prefix, nodes[cur].prefix, sizeof(uint16_t) * len);
        if (slot != 0) prefix[len++] = (uint16_t)alpha[slot - 1];
        const int32_t child = new_node(prefix, len, slot == 0);
        {
            auto& ch = nodes[cur].children;
            auto it = std::lower_bound(ch.begin(), ch.end(), std::make_pair(slot, (int32_t)-1));
            ch.insert(it, std::make_pair(slot, child));
        }
        path.push_back(child);
        // rollout
        if (slot != 0) {
            std::vector<int32_t> acts;
            for (;;) {
                slots(prefix, len, acts);
                const int32_t a = acts[(size_t)(draw() % (uint64_t)acts.size())];
                if (a == 0) break;
                prefix[len++] = (uint16_t)alpha[a - 1];
            }
        }
        // virtual loss, then the reward now or at tell time
        for (int32_t v : path) nodes[v].n += 1;
        const uint64_t code = code_of(prefix, len);
        auto hit = results.find(code);
        if (hit != results.end()) {
            const double r = reward(hit->second.first, hit->second.second);
            for (int32_t v : path) nodes[v].w += r;
        } else {
            auto wt = waiting.find(code);
            if (wt != waiting.end()) {
                wt->second.push_back(path);
            } else {
                pool.emplace_back(prefix, prefix + len);
                pool_codes.push_back(code);
                waiting[code].push_back(path);
            }
        }
        // exhaustion, bottom up
        for (size_t q = path.size(); q-- > 0;) {
            Node& v = nodes[path[q]];
            if (!v.untried.empty()) break;
            bool all = true;
            for (const auto& sc : v.children)
                if (!nodes[sc.second].exhausted) {
                    all = false;
                    break;
                }
            if (!all) break;
            v.exhausted = true;
        }
    }
};

namespace {

comet_status check_opts(const comet_mcts_opts* o) {
    if (!o) return mfail(COMET_ERR_INVALID_ARG, "mcts options are required");
    if (o->n_modes < 1 || o->n_modes > 65535) return mfail(COMET_ERR_INVALID_ARG, "mcts: n_modes out of range");
    if (o->l_max < 1 || o->l_max > COMET_MAX_SEGMENTS) return mfail(COMET_ERR_INVALID_ARG, "mcts: l_max out of range");
    unsigned __int128 p = 1;
    for (int i = 0; i <= o->l_max; ++i) {
        p *= (unsigned __int128)(o->n_modes + 1);
        if (p >> 64) return mfail(COMET_ERR_INVALID_ARG, "mcts: mode codes overflow 64 bits");
    }
    if (o->grammar != COMET_GRAMMAR_NONE && o->grammar != COMET_GRAMMAR_PUSH)
        return mfail(COMET_ERR_INVALID_ARG, "mcts: unknown grammar");
    if (o->grammar == COMET_GRAMMAR_PUSH && o->n_modes != 13)
        return mfail(COMET_ERR_INVALID_ARG, "mcts: the pushing grammar needs the 13-mode alphabet");
    if (o->reward != COMET_MCTS_REWARD_FEASIBLE && o->reward != COMET_MCTS_REWARD_MERIT)
        return mfail(COMET_ERR_INVALID_ARG, "mcts: unknown reward");
    if (!(o->c_uct >= 0.0) || !std::isfinite(o->c_uct)) return mfail(COMET_ERR_INVALID_ARG, "mcts: bad c_uct");
    if (o->max_evals < 0) return mfail(COMET_ERR_INVALID_ARG, "mcts: max_evals < 0");
    if (!(o->max_ms >= 0.0) || !std::isfinite(o->max_ms)) return mfail(COMET_ERR_INVALID_ARG, "mcts: bad max_ms");
    return COMET_OK;
}

}  // namespace

extern "C" {

comet_status comet_mcts_default_opts(comet_mcts_opts* o) {
    if (!o) return mfail(COMET_ERR_INVALID_ARG, "out is NULL");
    memset(o, 0, sizeof(*o));
    o->n_modes = 12;
    o->l_max = 4;
    o->grammar = COMET_GRAMMAR_NONE;
    o->reward = COMET_MCTS_REWARD_FEASIBLE;
    o->max_evals = 0;
    o->seed = 0;
    o->c_uct = 0.8;
    o->eps_feas = 1e-5;
    o->merit_mu = 100.0;
    o->max_ms = 0.0;
    return COMET_OK;
}

comet_status comet_mcts_create(const comet_mcts_opts* o, comet_mcts** out) {
    if (!out) return mfail(COMET_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    const comet_status st = check_opts(o);
    if (st != COMET_OK) return st;
    comet_mcts* t = new (std::nothrow) comet_mcts;
    if (!t) return mfail(COMET_ERR_OOM, "mcts: out of host memory");
    try {
        t->o = *o;
        if (o->grammar == COMET_GRAMMAR_PUSH)
            t->alpha = {0, 3, 6, 9, kPushFree};
        else
            for (int m = 0; m < o->n_modes; ++m) t->alpha.push_back(m);
        uint16_t none[1] = {0};
        t->new_node(none, 0, false);
    } catch (const std::bad_alloc&) {
        delete t;
        return mfail(COMET_ERR_OOM, "mcts: out of host memory");
    }
    *out = t;
    return COMET_OK;
}

comet_status comet_mcts_destroy(comet_mcts* t) {
    delete t;
    return COMET_OK;
}

comet_status comet_mcts_ask(comet_mcts* t, int32_t instance, int64_t pool, comet_mode_seq* out, int64_t* n) {
    if (!t || !out || !n || pool < 1) return mfail(COMET_ERR_INVALID_ARG, "mcts_ask: bad arguments");
    *n = 0;
    if (t->asked) return mfail(COMET_ERR_INVALID_ARG, "mcts_ask: tell the pending pool first");
    try {
        while ((int64_t)t->pool.size() < pool && !t->nodes[0].exhausted &&
               (t->o.max_evals <= 0 || t->issued + (int64_t)t->pool.size() < t->o.max_evals))
            t->attempt();
    } catch (const std::bad_alloc&) {
        return mfail(COMET_ERR_OOM, "mcts: out of host memory");
    }
    for (size_t i = 0; i < t->pool.size(); ++i) {
        comet_mode_seq q;
        memset(&q, 0, sizeof(q));
        q.instance = instance;
        q.len = (uint8_t)t->pool[i].size();
        for (size_t j = 0; j < t->pool[i].size(); ++j) q.modes[j] = t->pool[i][j];
        out[i] = q;
    }
    *n = (int64_t)t->pool.size();
    t->asked = *n > 0;
    return COMET_OK;
}

comet_status comet_mcts_tell(comet_mcts* t, const float* cost, const float* viol, int64_t n) {
    if (!t) return mfail(COMET_ERR_INVALID_ARG, "mcts_tell: search is NULL");
    if (!t->asked || n != (int64_t)t->pool.size()) return mfail(COMET_ERR_INVALID_ARG, "mcts_tell: not the pool's size");
    if (!cost || !viol) return mfail(COMET_ERR_INVALID_ARG, "mcts_tell: cost and viol are required");
    try {
        for (int64_t i = 0; i < n; ++i) {
            const double c = (double)cost[i], v = (double)viol[i];
            t->results[t->pool_codes[i]] = std::make_pair(c, v);
            t->result_codes.push_back(t->pool_codes[i]);
            t->best = std::min(t->best, t->value(c, v));
        }
    } catch (const std::bad_alloc&) {
        return mfail(COMET_ERR_OOM, "mcts: out of host memory");
    }
    for (int64_t i = 0; i < n; ++i) {
        const uint64_t code = t->pool_codes[i];
        const auto& res = t->results[code];
        const double r = t->reward(res.first, res.second);
        auto wt = t->waiting.find(code);
        for (const auto& path : wt->second)
            for (int32_t v : path) t->nodes[v].w += r;
        t->waiting.erase(wt);
    }
    t->issued += n;
    t->pool.clear();
    t->pool_codes.clear();
    t->asked = false;
    return COMET_OK;
}

comet_status comet_mcts_get_stats(const comet_mcts* t, comet_mcts_stats* out) {
    if (!t || !out) return mfail(COMET_ERR_INVALID_ARG, "mcts_get_stats: bad arguments");
    memset(out, 0, sizeof(*out));
    out->evaluations = t->issued;
    out->tree_nodes = (int64_t)t->nodes.size();
    out->pending = t->asked ? (int64_t)t->pool.size() : 0;
    out->exhausted = t->nodes[0].exhausted ? 1 : 0;
    out->best = t->best;
    return COMET_OK;
}

comet_status comet_mcts_best(const comet_mcts* t, int64_t k, uint64_t* codes, double* merits, int64_t* n) {
    if (!t || !codes || !n || k < 0) return mfail(COMET_ERR_INVALID_ARG, "mcts_best: bad arguments");
    std::vector<std::pair<double, uint64_t>> keys;
    keys.reserve(t->result_codes.size());
    for (uint64_t c : t->result_codes) {
        const auto& r = t->results.at(c);
        keys.emplace_back(t->merit(r.first, r.second), c);
    }
    const size_t m = (size_t)std::min<int64_t>(k, (int64_t)keys.size());
    std::partial_sort(keys.begin(), keys.begin() + (ptrdiff_t)m, keys.end());
    for (size_t i = 0; i < m; ++i) {
        codes[i] = keys[i].second;
        if (merits) merits[i] = keys[i].first;
    }
    *n = (int64_t)m;
    return COMET_OK;
}

comet_status comet_plan_mcts(comet_problem* p, int32_t instance, const comet_mcts_opts* o_in, int64_t pool,
                             const comet_plan_opts* po_in, comet_plan_result* out, float* out_traj) {
    if (!p || !o_in || !out || pool < 1) return mfail(COMET_ERR_INVALID_ARG, "plan_mcts: bad arguments");
    if (instance < 0 || instance >= (int32_t)p->inst.size()) return mfail(COMET_ERR_INVALID_ARG, "plan_mcts: bad instance");
    comet_plan_opts po;
    if (po_in)
        po = *po_in;
    else
        comet_default_plan_opts(&po);
    if (po.k_ref < 1) return mfail(COMET_ERR_INVALID_ARG, "plan_mcts: k_ref < 1");
    const comet_instance_desc& di = p->inst[instance];
    comet_mcts_opts o = *o_in;
    o.n_modes = di.n_modes;
    o.l_max = di.max_segments;
    o.eps_feas = p->opts.eps_feas;
    o.merit_mu = p->opts.merit_mu;
    comet_status st = check_opts(&o);
    if (st != COMET_OK) return st;
    if (o.max_evals == 0 && o.max_ms == 0.0) {
        // an unbounded search must end: the space has to be small
        double space = 0.0, pw = 1.0;
        for (int L = 1; L <= o.l_max; ++L) space += (pw *= (double)(o.grammar == COMET_GRAMMAR_PUSH ? 5 : o.n_modes));
        if (space > (double)(1 << 22)) return mfail(COMET_ERR_INVALID_ARG, "plan_mcts: set max_evals for this space");
    }
    comet_mcts* t = nullptr;
    st = comet_mcts_create(&o, &t);
    if (st != COMET_OK) return st;
    struct Guard {
        comet_mcts* t;
        ~Guard() { comet_mcts_destroy(t); }
    } guard{t};
    std::vector<comet_mode_seq> seqs;
    std::vector<float> cost, viol;
    std::vector<int32_t> status;
    try {
        seqs.resize((size_t)pool);
        cost.resize((size_t)pool);
        viol.resize((size_t)pool);
        status.resize((size_t)pool);
    } catch (const std::bad_alloc&) {
        return mfail(COMET_ERR_OOM, "plan_mcts: out of host memory");
    }
    const auto t0 = std::chrono::steady_clock::now();
    int32_t pools = 0;
    for (;;) {
        if (o.max_ms > 0.0 &&
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count() >= o.max_ms)
            break;
        int64_t n = 0;
        st = comet_mcts_ask(t, instance, pool, seqs.data(), &n);
        if (st != COMET_OK) return st;
        if (n == 0) break;
        st = comet_eval_modes(p, seqs.data(), n, nullptr, cost.data(), nullptr, status.data());
        if (st != COMET_OK) return st;
        st = comet_eval_stats(p, viol.data(), nullptr, nullptr, nullptr);
        if (st != COMET_OK) return st;
        st = comet_mcts_tell(t, cost.data(), viol.data(), n);
        if (st != COMET_OK) return st;
        ++pools;
    }
    const double search_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    comet_mcts_stats ms;
    comet_mcts_get_stats(t, &ms);
    if (ms.evaluations < 1) return mfail(COMET_ERR_INVALID_ARG, "plan_mcts: nothing was evaluated");
    // refinement as in Algorithm 1: the K_ref best orders by merit, re-solved
    // with t_ref (comet_plan with those orders as seeds and no round)
    std::vector<uint64_t> codes((size_t)po.k_ref);
    int64_t nb = 0;
    st = comet_mcts_best(t, po.k_ref, codes.data(), nullptr, &nb);
    if (st != COMET_OK) return st;
    std::vector<comet_mode_seq> top((size_t)nb);
    const uint64_t base = (uint64_t)o.n_modes + 1;
    for (int64_t i = 0; i < nb; ++i) {
        comet_mode_seq q;
        memset(&q, 0, sizeof(q));
        q.instance = instance;
        uint64_t c = codes[(size_t)i];
        q.len = (uint8_t)(c % base);
        c /= base;
        for (int j = 0; j < q.len; ++j) {
            q.modes[j] = (uint16_t)(c % base - 1);
            c /= base;
        }
        top[(size_t)i] = q;
    }
    comet_plan_opts pr = po;
    pr.rounds = 0;
    pr.budget = 0;
    pr.k_ref = (int32_t)nb;
    pr.batch = (int32_t)nb;
    pr.use_graph = 0;
    pr.radius = 1;
    pr.grammar = COMET_GRAMMAR_NONE;  // no expansion round runs
    st = comet_plan(p, instance, top.data(), nb, &pr, out, out_traj);
    if (st != COMET_OK) return st;
    out->evaluations = ms.evaluations;
    out->rounds_run = pools;
    out->explore_ms = (float)search_ms + out->explore_ms;
    return COMET_OK;
}

}  // extern "C"
