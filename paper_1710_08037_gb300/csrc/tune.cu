// tune.cu -- the autotuner of grouped plans (plv_group_tune) and the host-side
// layouts of a plan's two work lists.
//
// A grouped plan runs two kinds of persistent launches whose shapes are free
// choices that do not change any result:
//   - the any-length analytic-signal engine: which thread class (CTA width:
//     128 ... 1024 threads per transform, i.e. how many butterflies each
//     thread takes per stage) runs each transform length M, and how many
//     CTAs per SM each class launch keeps resident;
//   - the split-precision Gram: the order of its tile list, which is the
//     schedule, because CTA b of the persistent grid takes items b, b + G, ...
// The tuner times candidates of each on the plan's own buffers with CUDA
// events and keeps the fastest, then caches the choice in the handle under
// the plan's work signature so that an equal plan is configured without
// timing.  Every candidate computes the same values with the same
// arithmetic per transform and per tile; only the assignment of work to CTAs
// changes.
#include <algorithm>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "group.cuh"

namespace plv {

void k1_layout(const std::vector<K1Desc> &descs, const std::map<int, int> &cls,
               std::vector<int2> &items, K1Group &kg) {
    auto class_of = [&](int M) {
        auto it = cls.find(M);
        return it != cls.end() ? it->second : conv_class(M);
    };
    std::vector<int> order(descs.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const int ca = class_of(descs[a].plan.M), cb = class_of(descs[b].plan.M);
        if (ca != cb) return ca < cb;
        return descs[a].plan.M > descs[b].plan.M;
    });
    items.clear();
    for (int c = 0; c < kConvClasses; ++c) {
        kg.begin[c] = (int64_t)items.size();
        kg.max_M[c] = 0;
        for (int i : order) {
            if (class_of(descs[i].plan.M) != c) continue;
            kg.max_M[c] = std::max(kg.max_M[c], descs[i].plan.M);
            const int64_t pairs = (descs[i].rows + 1) / 2;
            for (int64_t pr = 0; pr < pairs; ++pr) items.push_back(make_int2(i, (int)pr));
        }
        kg.count[c] = (int64_t)items.size() - kg.begin[c];
    }
}

std::vector<int64_t> gram_order(const std::vector<int> &cost, int schedule, int G,
                                int tile_cost) {
    const int64_t n = (int64_t)cost.size();
    std::vector<int64_t> out(n);
    for (int64_t i = 0; i < n; ++i) out[i] = i;
    if (schedule == kSchedLongestFirst || G <= 1 || n <= G) return out;
    // Balanced rounds: deal the longest-first list in rounds of G items, each
    // round's items (longest first) to the CTAs with the least accumulated
    // cost (K blocks + tile_cost per item).  A CTA gets exactly one item per
    // full round, so the deal is a permutation within each round.  The
    // partial last round goes to the least-loaded CTAs, which are then
    // numbered 0 .. rem - 1 so that the round-robin launch gives them those
    // slots.
    const int64_t rounds = n / G, rem = n % G;
    std::vector<int64_t> load(G, 0);
    std::vector<std::vector<int64_t>> mine(G);  // per virtual CTA: indices into the list
    std::vector<int> ctas(G);
    for (int b = 0; b < G; ++b) ctas[b] = b;
    for (int64_t r = 0; r <= rounds; ++r) {
        const int64_t base = r * G;
        const int64_t cnt = r < rounds ? G : rem;
        if (cnt == 0) break;
        std::stable_sort(ctas.begin(), ctas.end(), [&](int a, int b) { return load[a] < load[b]; });
        for (int64_t k = 0; k < cnt; ++k) {
            const int b = ctas[k];
            const int64_t idx = base + k;
            mine[b].push_back(idx);
            load[b] += cost[idx] + tile_cost;
        }
    }
    // number the CTAs: those holding a last-round item first
    std::vector<int> label(G);
    std::vector<int> by_len(G);
    for (int b = 0; b < G; ++b) by_len[b] = b;
    std::stable_sort(by_len.begin(), by_len.end(), [&](int a, int b) {
        return mine[a].size() > mine[b].size();
    });
    for (int k = 0; k < G; ++k) label[by_len[k]] = k;
    for (int b = 0; b < G; ++b)
        for (size_t k = 0; k < mine[b].size(); ++k) out[(int64_t)k * G + label[b]] = mine[b][k];
    return out;
}

void split_plan(const std::vector<int> &nkb, int chunk, int G, int f, std::vector<int> &parts) {
    parts.assign(nkb.size(), 1);
    if (f <= 0 || G <= 0 || chunk <= 0) return;
    int64_t W = 0;
    for (int k : nkb) W += k;
    // a tile longer than L runs as parts of about L: the grid's fair share
    // / f, but at least kMinPartKb (a part's partial sums cost a 128 KB
    // round trip through L2) and a chunk
    const int64_t share = (W + (int64_t)G * f - 1) / ((int64_t)G * f);
    const int64_t L = std::max<int64_t>(std::max<int64_t>(chunk, kMinPartKb), share);
    std::vector<int> order(nkb.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return nkb[a] > nkb[b]; });
    int64_t slots = 0;
    for (int i : order) {
        const int64_t n = nkb[i];
        if (n <= L) break;
        const int64_t nch = (n + chunk - 1) / chunk;
        const int S = (int)std::min<int64_t>((n + L - 1) / L, nch);
        if (S < 2) continue;
        if (slots + S > kMaxSplitSlots) break;  // longest tiles first while slots last
        slots += S;
        parts[i] = S;
    }
}

void part_range(int nkb, int chunk, int S, int s, int &lo, int &hi) {
    const int64_t nch = (nkb + chunk - 1) / chunk;
    lo = (int)(chunk * ((int64_t)s * nch / S));
    hi = (int)std::min<int64_t>(nkb, chunk * ((int64_t)(s + 1) * nch / S));
}

GramList gram_list(const std::vector<TcProblem> &dp, const std::vector<int4> &tiles, int chunk,
                   int num_sms, const GroupConfig &cfg) {
    GramList L;
    std::vector<int> nkb(tiles.size());
    for (size_t i = 0; i < tiles.size(); ++i) nkb[i] = dp[tiles[i].x].nkb;
    std::vector<int> S;
    split_plan(nkb, chunk, num_sms, cfg.gram_split, S);
    // (tile, part) units; the parts of a tile get consecutive part numbers
    struct Unit {
        int tile, part, len;
    };
    std::vector<Unit> units;
    units.reserve(tiles.size());
    for (size_t i = 0; i < tiles.size(); ++i) {
        if (S[i] == 1) {
            units.push_back({(int)i, -1, nkb[i]});
            continue;
        }
        for (int s = 0; s < S[i]; ++s) {
            SplitPart p{};
            part_range(nkb[i], chunk, S[i], s, p.kb_lo, p.kb_hi);
            p.tile = L.ntiles;
            p.slot = L.nslots + s;
            p.s = s;
            p.S = S[i];
            units.push_back({(int)i, (int)L.parts.size(), p.kb_hi - p.kb_lo});
            L.parts.push_back(p);
        }
        L.nslots += S[i];
        ++L.ntiles;
    }
    // longest first, then the schedule
    std::stable_sort(units.begin(), units.end(),
                     [](const Unit &a, const Unit &b) { return a.len > b.len; });
    std::vector<int> cost(units.size());
    for (size_t k = 0; k < units.size(); ++k) cost[k] = units[k].len;
    const int G = (int64_t)units.size() < num_sms ? (int)units.size() : num_sms;
    const std::vector<int64_t> order = gram_order(cost, cfg.gram_schedule, G, cfg.gram_tile_cost);
    L.items.resize(units.size());
    for (size_t k = 0; k < units.size(); ++k) {
        const Unit &u = units[order[k]];
        const int4 &t = tiles[u.tile];
        L.items[k] = make_int4(t.x, t.y, t.z | (t.w << 16), u.part + 1);
    }
    return L;
}

bool covers(const std::vector<TcProblem> &dp, const std::vector<int4> &tiles,
            const GramList &list) {
    // every tile's K range, as the union of its entries' ranges, exactly once
    std::map<std::tuple<int, int, int, int>, std::vector<std::pair<int, int>>> got;
    for (const int4 &it : list.items) {
        const int I = it.z & 0xffff, J = (int)((unsigned)it.z >> 16);
        if (it.x < 0 || it.x >= (int)dp.size()) return false;
        int lo = 0, hi = dp[it.x].nkb;
        if (it.w > 0) {
            if (it.w - 1 >= (int)list.parts.size()) return false;
            const SplitPart &p = list.parts[it.w - 1];
            if (p.s < 0 || p.s >= p.S || p.slot - p.s < 0 || p.slot - p.s + p.S > list.nslots ||
                p.tile < 0 || p.tile >= list.ntiles)
                return false;
            lo = p.kb_lo;
            hi = p.kb_hi;
        }
        got[std::make_tuple(it.x, it.y, I, J)].push_back({lo, hi});
    }
    if (got.size() != tiles.size()) return false;
    for (const int4 &t : tiles) {
        auto f = got.find(std::make_tuple(t.x, t.y, t.z, t.w));
        if (f == got.end()) return false;
        auto r = f->second;
        std::sort(r.begin(), r.end());
        int at = 0;
        for (auto &pr : r) {
            if (pr.first != at || pr.second <= pr.first) return false;
            at = pr.second;
        }
        if (at != dp[t.x].nkb) return false;
    }
    return true;
}

plv_status upload_list(const GramList &list, cudaStream_t s, int4 **items, TcSplit *split) {
    *items = nullptr;
    *split = TcSplit{};
    int4 *di = nullptr;
    SplitPart *dparts = nullptr;
    float *dslots = nullptr;
    int *dcnt = nullptr;
    plv_status st = check_alloc(dev_malloc(&di, sizeof(int4) * std::max<size_t>(list.items.size(), 1)),
                                "gram work list");
    if (st == PLV_OK && !list.parts.empty())
        st = check_alloc(dev_malloc(&dparts, sizeof(SplitPart) * list.parts.size()),
                         "split parts");
    if (st == PLV_OK && list.nslots > 0)
        st = check_alloc(dev_malloc(&dslots, sizeof(float) * (size_t)kTileFloats * list.nslots),
                         "split slots");
    if (st == PLV_OK && list.ntiles > 0)
        st = check_alloc(dev_malloc(&dcnt, sizeof(int) * 16 * (size_t)list.ntiles),
                         "split counters");
    if (st == PLV_OK)
        st = check_cuda(cudaMemcpyAsync(di, list.items.data(), sizeof(int4) * list.items.size(),
                                        cudaMemcpyHostToDevice, s),
                        "gram work list upload");
    if (st == PLV_OK && dparts)
        st = check_cuda(cudaMemcpyAsync(dparts, list.parts.data(),
                                        sizeof(SplitPart) * list.parts.size(),
                                        cudaMemcpyHostToDevice, s),
                        "split parts upload");
    if (st == PLV_OK && dcnt)
        st = check_cuda(cudaMemsetAsync(dcnt, 0, sizeof(int) * 16 * (size_t)list.ntiles, s),
                        "split counters");
    if (st == PLV_OK) st = check_cuda(cudaStreamSynchronize(s), "gram work list upload");
    if (st != PLV_OK) {
        if (di) cudaFree(di);
        if (dparts) cudaFree(dparts);
        if (dslots) cudaFree(dslots);
        if (dcnt) cudaFree(dcnt);
        return st;
    }
    *items = di;
    split->parts = dparts;
    split->partials = dslots;
    split->counters = dcnt;
    split->nslots = list.nslots;
    split->ntiles = list.ntiles;
    return PLV_OK;
}

void free_list(int4 *items, const TcSplit &split) {
    if (items) cudaFree(items);
    if (split.parts) cudaFree((void *)split.parts);
    if (split.partials) cudaFree(split.partials);
    if (split.counters) cudaFree(split.counters);
}

namespace {

// Work signature of a plan: precision, SM count, the (M, row pairs) of its
// transforms and the (K blocks, tiles) of its Gram.
std::string signature(const Handle &h, const plv_group &g) {
    std::map<int, int64_t> k1;
    for (const K1Desc &d : g.k1_host) k1[d.plan.M] += (d.rows + 1) / 2;
    std::map<int, int64_t> gram;
    for (const int4 &it : g.items_host) gram[g.dp_host[it.x].nkb] += 1;
    std::string s = "p" + std::to_string((int)h.prec) + "s" + std::to_string(h.num_sms) + "|";
    for (auto &kv : k1) s += std::to_string(kv.first) + ":" + std::to_string(kv.second) + ",";
    s += "|";
    for (auto &kv : gram) s += std::to_string(kv.first) + ":" + std::to_string(kv.second) + ",";
    return s;
}

// Median of `reps` timed runs of fn on stream s (after one untimed run).
template <class F>
plv_status time_median(cudaStream_t s, int reps, F fn, float *ms) {
    cudaEvent_t a = nullptr, b = nullptr;
    plv_status st = check_cuda(cudaEventCreate(&a), "plv_group_tune: event");
    if (st == PLV_OK) st = check_cuda(cudaEventCreate(&b), "plv_group_tune: event");
    std::vector<float> t;
    if (st == PLV_OK) st = check_cuda(fn(), "plv_group_tune: launch");
    for (int r = 0; r < reps && st == PLV_OK; ++r) {
        st = check_cuda(cudaEventRecord(a, s), "plv_group_tune: record");
        if (st == PLV_OK) st = check_cuda(fn(), "plv_group_tune: launch");
        if (st == PLV_OK) st = check_cuda(cudaEventRecord(b, s), "plv_group_tune: record");
        if (st == PLV_OK) st = check_cuda(cudaEventSynchronize(b), "plv_group_tune: wait");
        float v = 0.f;
        if (st == PLV_OK) st = check_cuda(cudaEventElapsedTime(&v, a, b), "plv_group_tune: time");
        t.push_back(v);
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (st != PLV_OK) return st;
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    return PLV_OK;
}

// A fresh device copy of a host list.  Lists are never rewritten in place:
// graphs captured earlier keep the arrays their launches were captured with.
template <class T>
plv_status upload(const std::vector<T> &v, T **out, cudaStream_t s) {
    T *d = nullptr;
    plv_status st = check_alloc(dev_malloc(&d, sizeof(T) * std::max<size_t>(v.size(), 1)),
                               "plv_group_tune: work list");
    if (st != PLV_OK) return st;
    st = check_cuda(cudaMemcpyAsync(d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, s),
                    "plv_group_tune: upload");
    if (st == PLV_OK) st = check_cuda(cudaStreamSynchronize(s), "plv_group_tune: upload");
    if (st != PLV_OK) {
        cudaFree(d);
        return st;
    }
    *out = d;
    return PLV_OK;
}

// CTAs per SM a class launch gets from its register budget alone.
int k1_default_per_sm(int c) {
    const int v = 65536 / (kConvRegs * conv_class_threads(c));
    return v > 0 ? v : 1;
}

// Make cfg the plan's configuration: new device lists, the old ones retired
// (nothing to do when the plan already runs cfg).
plv_status apply_config(const Handle &h, plv_group &g, const GroupConfig &cfg, cudaStream_t s) {
    if (cfg == g.cfg) return PLV_OK;
    if (g.has_k1) {
        std::vector<int2> items;
        K1Group kg = g.k1;
        k1_layout(g.k1_host, cfg.k1_class, items, kg);
        for (int c = 0; c < kConvClasses; ++c) kg.per_sm[c] = cfg.k1_per_sm[c];
        int2 *d = nullptr;
        plv_status st = upload(items, &d, s);
        if (st != PLV_OK) return st;
        g.retired.push_back(g.k1_items);
        g.k1_items = d;
        kg.items = d;
        g.k1 = kg;
    }
    if (g.prec != PLV_PREC_FP32 && g.ntiles > 0) {
        const GramList list =
            gram_list(g.dp_host, g.items_host, gram_chunk_kb(g.prec), h.num_sms, cfg);
        if (!covers(g.dp_host, g.items_host, list))
            return fail(PLV_ERR_NUMERIC, "plv_group_tune: internal error: the launch list does "
                                         "not cover every tile once");
        int4 *d = nullptr;
        TcSplit sp;
        plv_status st = upload_list(list, s, &d, &sp);
        if (st != PLV_OK) return st;
        g.retired.push_back(g.items);
        g.retired.push_back((void *)g.split.parts);
        g.retired.push_back(g.split.partials);
        g.retired.push_back(g.split.counters);
        g.items = d;
        g.split = sp;
        g.nitems = (int)list.items.size();
    }
    g.cfg = cfg;
    return PLV_OK;
}

}  // namespace
}  // namespace plv

using namespace plv;

extern "C" plv_status plv_group_tune(plv_handle *hp, void *stream, plv_group *g, int reps,
                                     plv_tune_result *res) {
    PLV_RANGE("plv_group_tune");
    if (!hp || !g) return fail(PLV_ERR_INVALID, "plv_group_tune: NULL argument");
    Handle &h = hp->h;
    if (g->device != h.device || g->prec != h.prec)
        return fail(PLV_ERR_INVALID, "plv_group_tune: plan made for another device or precision");
    if (reps < 1 || reps > 100)
        return fail(PLV_ERR_INVALID, "plv_group_tune: reps = %d (1..100)", reps);
    DeviceGuard guard(h.device);
    if (!guard.ok) return fail(PLV_ERR_CUDA, "cannot select device %d", h.device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        return fail(PLV_ERR_INVALID, "plv_group_tune: the stream is capturing (tuning times "
                                     "launches and allocates)");
    plv_tune_result r{};
    const bool gram = g->prec != PLV_PREC_FP32 && g->nitems > 0;
    std::vector<int> lengths;
    for (const K1Desc &d : g->k1_host)
        if (std::find(lengths.begin(), lengths.end(), d.plan.M) == lengths.end())
            lengths.push_back(d.plan.M);
    std::sort(lengths.begin(), lengths.end(), std::greater<int>());
    r.k1_lengths = (int)lengths.size();
    const std::string sig = signature(h, *g);
    plv_status st = check_cuda(cudaDeviceSynchronize(), "plv_group_tune: synchronise");
    if (st != PLV_OK) return st;

    GroupConfig cfg;
    bool cached = false;
    {
        std::lock_guard<std::mutex> lock(h.mu);
        auto it = h.tuned.find(sig);
        if (it != h.tuned.end()) {
            cfg = it->second;
            cached = true;
        }
    }
    auto run_k1 = [&](const K1Group &kg) {
        return launch_analytic_group(&h, s, g->k1_dtype, kg);
    };
    auto run_gram = [&](const int4 *items, int n, const TcSplit &sp) {
        cudaError_t e = cudaSuccess;
        if (g->any_diag) e = launch_zero_group_diag(s, g->probs, g->nprob);
        if (e == cudaSuccess && sp.ntiles > 0)
            e = cudaMemsetAsync(sp.counters, 0, sizeof(int) * 16 * (size_t)sp.ntiles, s);
        if (e == cudaSuccess) e = launch_gram_tc_group(&h, s, g->probs, items, n, sp);
        return e;
    };
    // the Gram's launch list under configuration c, timed
    auto time_gram = [&](const GroupConfig &c, float *ms) {
        const GramList list =
            gram_list(g->dp_host, g->items_host, gram_chunk_kb(g->prec), h.num_sms, c);
        if (!covers(g->dp_host, g->items_host, list))
            return fail(PLV_ERR_NUMERIC, "plv_group_tune: internal error: the launch list does "
                                         "not cover every tile once");
        int4 *d = nullptr;
        TcSplit sp;
        plv_status st2 = upload_list(list, s, &d, &sp);
        if (st2 != PLV_OK) return st2;
        st2 = time_median(s, reps, [&] { return run_gram(d, (int)list.items.size(), sp); }, ms);
        cudaStreamSynchronize(s);
        free_list(d, sp);
        return st2;
    };

    if (!cached && g->has_k1) {
        // 1. default configuration
        K1Group base = g->k1;
        st = time_median(s, reps, [&] { return run_k1(base); }, &r.k1_ms_default);
        ++r.timed_configs;
        // 2. thread class of each transform length: its own or the next
        //    wider one, timed on that length's items alone
        std::vector<int2> by_m;
        std::vector<std::pair<int64_t, int64_t>> range;
        for (int M : lengths) {
            const int64_t b = (int64_t)by_m.size();
            for (size_t i = 0; i < g->k1_host.size(); ++i) {
                if (g->k1_host[i].plan.M != M) continue;
                const int64_t pairs = (g->k1_host[i].rows + 1) / 2;
                for (int64_t pr = 0; pr < pairs; ++pr) by_m.push_back(make_int2((int)i, (int)pr));
            }
            range.push_back({b, (int64_t)by_m.size() - b});
        }
        int2 *d_by_m = nullptr;
        if (st == PLV_OK) st = upload(by_m, &d_by_m, s);
        for (size_t li = 0; li < lengths.size() && st == PLV_OK; ++li) {
            const int M = lengths[li];
            const int c0 = conv_class(M);
            int best = c0;
            float best_ms = 0.f;
            for (int c = c0; c <= std::min(c0 + 1, kConvClasses - 1) && st == PLV_OK; ++c) {
                K1Group kg{};
                kg.descs = g->k1_descs;
                kg.items = d_by_m;
                kg.begin[c] = range[li].first;
                kg.count[c] = range[li].second;
                kg.max_M[c] = M;
                float ms = 0.f;
                st = time_median(s, reps, [&] { return run_k1(kg); }, &ms);
                ++r.timed_configs;
                if (c == c0 || ms < 0.97f * best_ms) {
                    best = c;
                    best_ms = ms;
                }
            }
            if (best != c0) {
                cfg.k1_class[M] = best;
                ++r.k1_widened;
            }
        }
        if (d_by_m) {
            cudaStreamSynchronize(s);
            cudaFree(d_by_m);
        }
        // 3. CTAs per SM of each class launch in the chosen layout
        std::vector<int2> items;
        K1Group lay = g->k1;
        if (st == PLV_OK) k1_layout(g->k1_host, cfg.k1_class, items, lay);
        int2 *d_items = nullptr;
        if (st == PLV_OK) st = upload(items, &d_items, s);
        lay.items = d_items;
        for (int c = 0; c < kConvClasses && st == PLV_OK; ++c) {
            lay.per_sm[c] = 0;
            if (lay.count[c] == 0) continue;
            K1Group one = lay;
            for (int o = 0; o < kConvClasses; ++o)
                if (o != c) one.count[o] = 0;
            float best_ms = 0.f;
            int best = 0;
            for (int k = 0; st == PLV_OK; ++k) {
                const int ps = k == 0 ? 0 : k1_default_per_sm(c) >> k;
                if (k > 0 && ps < 1) break;
                one.per_sm[c] = ps;
                float ms = 0.f;
                st = time_median(s, reps, [&] { return run_k1(one); }, &ms);
                ++r.timed_configs;
                if (k == 0 || ms < 0.97f * best_ms) {
                    best = ps;
                    best_ms = ms;
                }
            }
            cfg.k1_per_sm[c] = best;
            lay.per_sm[c] = best;
        }
        // 4. the whole tuned configuration; keep the default if it is not faster
        float tuned_ms = 0.f;
        if (st == PLV_OK) st = time_median(s, reps, [&] { return run_k1(lay); }, &tuned_ms);
        ++r.timed_configs;
        if (d_items) {
            cudaStreamSynchronize(s);
            cudaFree(d_items);
        }
        if (st == PLV_OK && tuned_ms >= r.k1_ms_default) {
            cfg.k1_class.clear();
            for (int c = 0; c < kConvClasses; ++c) cfg.k1_per_sm[c] = 0;
            r.k1_widened = 0;
            tuned_ms = r.k1_ms_default;
        }
        r.k1_ms_tuned = tuned_ms;
        if (st != PLV_OK) return st;
    }

    if (!cached && gram) {
        // P holds valid phasors (step 1 wrote them, or the caller did).
        // 1. the default: longest first, no tile split
        GroupConfig best = cfg;
        best.gram_schedule = kSchedLongestFirst;
        best.gram_tile_cost = 0;
        best.gram_split = 0;
        st = time_gram(best, &r.gram_ms_default);
        ++r.timed_configs;
        float best_ms = r.gram_ms_default;
        // 2. the schedule: balanced rounds under per-tile costs
        const GroupConfig plain = best;
        for (int cost : {0, 8, 32}) {
            if (st != PLV_OK) break;
            GroupConfig c = plain;
            c.gram_schedule = kSchedBalanced;
            c.gram_tile_cost = cost;
            float ms = 0.f;
            st = time_gram(c, &ms);
            ++r.timed_configs;
            if (st == PLV_OK && ms < 0.99f * best_ms) {
                best_ms = ms;
                best = c;
            }
        }
        // 3. split K of the longest tiles, in the chosen schedule (factors
        //    whose split plan splits no tile are the unsplit list: skipped)
        const GroupConfig sched = best;
        const float sched_ms = best_ms;
        for (int f : {1, 2, 4}) {
            if (st != PLV_OK) break;
            GroupConfig c = sched;
            c.gram_split = f;
            if (gram_list(g->dp_host, g->items_host, gram_chunk_kb(g->prec), h.num_sms, c)
                    .ntiles == 0)
                continue;
            float ms = 0.f;
            st = time_gram(c, &ms);
            ++r.timed_configs;
            if (st == PLV_OK && ms < 0.97f * sched_ms && ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
        cfg.gram_schedule = best.gram_schedule;
        cfg.gram_tile_cost = best.gram_tile_cost;
        cfg.gram_split = best.gram_split;
        r.gram_ms_tuned = best_ms;
        if (st != PLV_OK) return st;
    }

    st = apply_config(h, *g, cfg, s);
    if (st != PLV_OK) return st;
    if (!cached) {
        std::lock_guard<std::mutex> lock(h.mu);
        h.tuned[sig] = cfg;
    }
    r.k1_widened = (int)cfg.k1_class.size();
    for (int c = 0; c < kConvClasses; ++c) {
        r.k1_per_sm[c] = cfg.k1_per_sm[c];
        if (g->has_k1 && g->k1.count[c] > 0) ++r.k1_launches;
    }
    r.gram_schedule = cfg.gram_schedule;
    r.gram_tile_cost = cfg.gram_tile_cost;
    r.gram_split = cfg.gram_split;
    r.gram_split_tiles = g->split.ntiles;
    r.cached = cached ? 1 : 0;
    if (res) *res = r;
    return PLV_OK;
}

extern "C" plv_status plv_group_configure(plv_handle *hp, void *stream, plv_group *g,
                                          int k1_widen, const int *k1_per_sm,
                                          int gram_schedule, int gram_tile_cost,
                                          int gram_split) {
    PLV_RANGE("plv_group_configure");
    if (!hp || !g) return fail(PLV_ERR_INVALID, "plv_group_configure: NULL argument");
    Handle &h = hp->h;
    if (g->device != h.device || g->prec != h.prec)
        return fail(PLV_ERR_INVALID,
                    "plv_group_configure: plan made for another device or precision");
    if (k1_widen != 0 && k1_widen != 1)
        return fail(PLV_ERR_INVALID, "plv_group_configure: k1_widen = %d (0 or 1)", k1_widen);
    if (gram_schedule != kSchedLongestFirst && gram_schedule != kSchedBalanced)
        return fail(PLV_ERR_INVALID, "plv_group_configure: gram_schedule = %d (0 or 1)",
                    gram_schedule);
    if (gram_tile_cost < 0 || gram_tile_cost > (1 << 20))
        return fail(PLV_ERR_INVALID, "plv_group_configure: gram_tile_cost = %d", gram_tile_cost);
    if (gram_split < 0 || gram_split > kMaxSplitFactor)
        return fail(PLV_ERR_INVALID, "plv_group_configure: gram_split = %d (0..%d)", gram_split,
                    kMaxSplitFactor);
    GroupConfig cfg;
    for (int c = 0; c < kConvClasses; ++c) {
        const int v = k1_per_sm ? k1_per_sm[c] : 0;
        if (v < 0 || v > 64)
            return fail(PLV_ERR_INVALID, "plv_group_configure: k1_per_sm[%d] = %d (0..64)", c, v);
        cfg.k1_per_sm[c] = v;
    }
    if (k1_widen)
        for (const K1Desc &d : g->k1_host) {
            const int c = conv_class(d.plan.M);
            if (c + 1 < kConvClasses) cfg.k1_class[d.plan.M] = c + 1;
        }
    cfg.gram_schedule = gram_schedule;
    cfg.gram_tile_cost = gram_tile_cost;
    cfg.gram_split = gram_split;
    DeviceGuard guard(h.device);
    if (!guard.ok) return fail(PLV_ERR_CUDA, "cannot select device %d", h.device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        return fail(PLV_ERR_INVALID, "plv_group_configure: the stream is capturing");
    plv_status st = check_cuda(cudaDeviceSynchronize(), "plv_group_configure: synchronise");
    if (st != PLV_OK) return st;
    return apply_config(h, *g, cfg, s);
}

extern "C" plv_status plv_gram_split_plan(const int *nkb, int ntiles, int chunk, int grid,
                                          int split, int *parts) {
    if (ntiles < 0 || (ntiles > 0 && (!nkb || !parts)))
        return fail(PLV_ERR_INVALID, "plv_gram_split_plan: bad tile list");
    if (chunk < 1 || grid < 1 || split < 0 || split > kMaxSplitFactor)
        return fail(PLV_ERR_INVALID, "plv_gram_split_plan: chunk %d, grid %d, split %d", chunk,
                    grid, split);
    std::vector<int> k(nkb, nkb + ntiles), S;
    for (int v : k)
        if (v < 1) return fail(PLV_ERR_INVALID, "plv_gram_split_plan: tile of %d K blocks", v);
    split_plan(k, chunk, grid, split, S);
    for (int i = 0; i < ntiles; ++i) parts[i] = S[i];
    return PLV_OK;
}
