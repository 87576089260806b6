"""Host-side logic of the library on CPU, through small C++ programs linked
against the built library (pure host functions: no GPU needed):
- the autotuner's work lists: plv::gram_order (the grouped Gram's tile
  schedules), plv::gram_list with split K (parts of whole chunks covering
  every tile once, their slots and counters), plv::tile_raster (the
  single-problem Gram's tile order: a permutation of the upper triangle for
  every width) and plv::k1_layout (the grouped analytic signal's items by
  thread class);
- the any-length plans: the transform length for T, its radix order, and
  the FP64 inverse DFT of any length that builds the band kernels, against
  a direct sum."""
import os
import shutil
import subprocess

import pytest

from paper_1710_08037_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <cstdio>
#include <cstdlib>
#include <map>
#include <tuple>
#include <vector>
#include <algorithm>
#include "group.cuh"
using namespace plv;

#define CHECK(c) do { if (!(c)) { std::printf("FAIL %s:%d %s\n", __FILE__, __LINE__, #c); \
    return 1; } } while (0)

static std::vector<long> loads(const std::vector<int> &cost, const std::vector<int64_t> &o,
                               int G, int c0) {
    std::vector<long> l(G, 0);
    for (size_t t = 0; t < o.size(); ++t) l[t % G] += cost[o[t]] + c0;
    return l;
}

int main() {
    // grouped Gram: problems of different K lengths, tiles longest first
    const int nkb[5] = {313, 160, 40, 16, 3}, cnt[5] = {300, 200, 517, 100, 37};
    std::vector<TcProblem> dp(5);
    std::vector<int4> items;
    std::vector<int> cost;
    for (int p = 0; p < 5; ++p) {
        dp[p] = TcProblem{};
        dp[p].nkb = nkb[p];
        for (int c = 0; c < cnt[p]; ++c) {
            items.push_back(make_int4(p, c, 0, 0));
            cost.push_back(nkb[p]);
        }
    }
    const int64_t n = (int64_t)items.size();
    for (int G : {1, 7, 152, 2000}) {
        CHECK((int64_t)gram_order(cost, 0, G, 0).size() == n);
        const std::vector<long> base = loads(cost, gram_order(cost, 0, G, 0), G, 0);
        for (int c0 : {0, 8, 32}) {
            const std::vector<int64_t> o = gram_order(cost, 1, G, c0);
            // a permutation of the list
            std::vector<int64_t> s = o;
            std::sort(s.begin(), s.end());
            for (int64_t i = 0; i < n; ++i) CHECK(s[i] == i);
            // no CTA's K-block load is further from the mean than under longest first
            const std::vector<long> lb = loads(cost, o, G, 0);
            const long spread = *std::max_element(lb.begin(), lb.end()) -
                                *std::min_element(lb.begin(), lb.end());
            const long spread0 = *std::max_element(base.begin(), base.end()) -
                                 *std::min_element(base.begin(), base.end());
            if (c0 == 0) CHECK(spread <= spread0);
            // each round of G slots holds the entries of one longest-first round
            for (size_t r = 0; r * G < o.size(); ++r) {
                const size_t b = r * G, e = std::min(o.size(), b + (size_t)G);
                std::vector<int64_t> a(o.begin() + b, o.begin() + e);
                std::sort(a.begin(), a.end());
                for (size_t i = 0; i < a.size(); ++i) CHECK(a[i] == (int64_t)(b + i));
            }
        }
    }
    // longest first is the list as given
    {
        const std::vector<int64_t> o = gram_order(cost, 0, 152, 0);
        for (int64_t i = 0; i < n; ++i) CHECK(o[i] == i);
    }
    // the launch list: tiles (problem, epoch, I, J) with I <= J, longest first
    {
        std::vector<int4> tiles;
        const int nrb[5] = {3, 1, 2, 1, 4};
        for (int p = 0; p < 5; ++p)
            for (int e = 0; e < 2; ++e)
                for (int J = 0; J < nrb[p]; ++J)
                    for (int I = 0; I <= J; ++I) tiles.push_back(make_int4(p, e, I, J));
        std::stable_sort(tiles.begin(), tiles.end(), [&](const int4 &a, const int4 &b) {
            return dp[a.x].nkb > dp[b.x].nkb;
        });
        for (int chunk : {4, 16})
            for (int f : {0, 1, 2, 4, 64})
                for (int sched : {0, 1}) {
                    GroupConfig cfg;
                    cfg.gram_split = f;
                    cfg.gram_schedule = sched;
                    cfg.gram_tile_cost = 8;
                    const GramList L = gram_list(dp, tiles, chunk, 152, cfg);
                    CHECK(covers(dp, tiles, L));
                    if (f == 0) CHECK(L.parts.empty() && L.items.size() == tiles.size());
                    // parts: whole chunks, at least 64 K blocks unless the tile's end,
                    // consecutive slots per tile, one counter per split tile
                    std::map<int, std::vector<SplitPart>> by_tile;
                    for (const SplitPart &q : L.parts) by_tile[q.tile].push_back(q);
                    CHECK((int)by_tile.size() == L.ntiles);
                    int slots = 0;
                    for (auto &kv : by_tile) {
                        const std::vector<SplitPart> &v = kv.second;
                        CHECK((int)v.size() == v[0].S && v[0].S >= 2);
                        for (int s2 = 0; s2 < (int)v.size(); ++s2) {
                            CHECK(v[s2].s == s2 && v[s2].S == v[0].S);
                            CHECK(v[s2].slot == v[0].slot + s2);
                            CHECK(v[s2].kb_lo % chunk == 0);
                            if (s2 + 1 < (int)v.size()) CHECK(v[s2].kb_hi == v[s2 + 1].kb_lo);
                            CHECK(v[s2].kb_hi - v[s2].kb_lo >= std::min(64, chunk));
                        }
                        slots += v[0].S;
                    }
                    CHECK(slots == L.nslots);
                    // the launch list is longest first under longest-first scheduling
                    if (sched == 0)
                        for (size_t i = 1; i < L.items.size(); ++i) {
                            auto len = [&](const int4 &it) {
                                return it.w ? L.parts[it.w - 1].kb_hi - L.parts[it.w - 1].kb_lo
                                            : dp[it.x].nkb;
                            };
                            CHECK(len(L.items[i - 1]) >= len(L.items[i]));
                        }
                }
        // a long tile split at f = 1 in a short plan: 313 K blocks, parts of >= 64
        GroupConfig cfg;
        cfg.gram_split = 1;
        std::vector<int4> one(1, make_int4(0, 0, 0, 0));
        const GramList L = gram_list(dp, one, 16, 152, cfg);
        CHECK(L.parts.size() == 5 && L.ntiles == 1 && L.nslots == 5);
        CHECK(L.parts[0].kb_lo == 0 && L.parts[4].kb_hi == 313);
    }
    // the single-problem tile raster: for every width and triangle size, a
    // permutation of the upper-triangle tiles, each super-column of W block
    // columns before the next, and the plain column-major triangle when W >= nrb
    for (int nrb = 1; nrb <= 70; ++nrb)
        for (int W = 1; W <= 20; ++W) {
            const int n = nrb * (nrb + 1) / 2;
            std::vector<char> seen((size_t)nrb * nrb, 0);
            int prev_sj = 0;
            for (int t = 0; t < n; ++t) {
                int I = -1, J = -1;
                tile_raster(t, nrb, W, I, J);
                CHECK(0 <= I && I <= J && J < nrb);
                CHECK(!seen[(size_t)I * nrb + J]);
                seen[(size_t)I * nrb + J] = 1;
                CHECK(J / W >= prev_sj);
                prev_sj = J / W;
                if (W >= nrb) {
                    int I0, J0;
                    upper_tile_of(t, I0, J0);
                    CHECK(I0 == I && J0 == J);
                }
            }
        }
    // grouped analytic signal: problems with transform lengths in all classes
    const int Ms[6] = {1280, 20480, 4096, 1280, 10240, 768};
    const long rows[6] = {70, 40, 201, 1, 130, 9};
    std::vector<K1Desc> descs(6);
    for (int i = 0; i < 6; ++i) {
        descs[i] = K1Desc{};
        descs[i].plan.M = Ms[i];
        descs[i].rows = rows[i];
    }
    for (int widen = 0; widen < 2; ++widen) {
        std::map<int, int> cls;
        if (widen)
            for (int i = 0; i < 6; ++i)
                if (conv_class(Ms[i]) < kConvClasses - 1) cls[Ms[i]] = conv_class(Ms[i]) + 1;
        std::vector<int2> it;
        K1Group kg{};
        k1_layout(descs, cls, it, kg);
        long total = 0;
        for (int i = 0; i < 6; ++i) total += (rows[i] + 1) / 2;
        CHECK((long)it.size() == total);
        long seen = 0;
        for (int c = 0; c < kConvClasses; ++c) {
            CHECK(kg.begin[c] == seen);
            int prevM = 1 << 30, maxM = 0;
            for (long k = kg.begin[c]; k < kg.begin[c] + kg.count[c]; ++k) {
                const int M = descs[it[k].x].plan.M;
                const int want = cls.count(M) ? cls[M] : conv_class(M);
                CHECK(want == c);                       // in its assigned class
                CHECK(M <= prevM);                      // longest transform first
                CHECK(M <= conv_class_max_M(c));        // fits the class's buffer
                CHECK(it[k].y >= 0 && it[k].y < (rows[it[k].x] + 1) / 2);
                prevM = M;
                maxM = std::max(maxM, M);
            }
            CHECK(kg.max_M[c] == maxM);
            seen += kg.count[c];
        }
        CHECK(seen == total);
    }
    std::printf("ok\n");
    return 0;
}
"""


PLAN_PROGRAM = r"""
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "common.cuh"
namespace plv {
int conv_length(int T);
std::vector<int> conv_radix_order(int M);
std::vector<std::complex<double>> inverse_dft_any(const std::vector<std::complex<double>> &Y);
}
using namespace plv;
typedef std::complex<double> cd;

#define CHECK(c) do { if (!(c)) { std::printf("FAIL %s:%d %s\n", __FILE__, __LINE__, #c); \
    return 1; } } while (0)

int main() {
    for (int T = 2; T <= kMaxConvM / 2; T += (T < 300 ? 1 : 97)) {
        const int M = conv_length(T);
        // the smallest 2^a, 3 2^a or 5 2^a (>= 32) that holds 2T - 1
        CHECK(M >= 2 * T - 1 && M >= 32 && M <= kMaxConvM);
        int odd = M;
        while (odd % 2 == 0) odd /= 2;
        CHECK(odd == 1 || odd == 3 || odd == 5);
        for (int f : {1, 3, 5})
            for (int p = 32; f * p < M; p *= 2) CHECK(f * p < 2 * T - 1);
        // radix order: stages of at most kConvMaxRadix whose product is M, the
        // odd factor (if any) first so that every later span is a power of two
        const std::vector<int> r = conv_radix_order(M);
        CHECK(!r.empty() && (int)r.size() <= 8);
        long prod = 1;
        for (size_t k = 0; k < r.size(); ++k) {
            CHECK(r[k] >= 2 && r[k] <= kConvMaxRadix);
            if (k > 0) CHECK((r[k] & (r[k] - 1)) == 0);
            prod *= r[k];
        }
        CHECK(prod == M);
        if (odd != 1) CHECK(r[0] == odd);
    }
    // FP64 inverse DFT of any length against the direct sum
    for (int T : {1, 2, 3, 5, 7, 31, 100, 333, 1000, 4097, 12288}) {
        std::vector<cd> Y(T);
        std::srand(T);
        for (int k = 0; k < T; ++k)
            Y[k] = cd(std::rand() / (double)RAND_MAX - 0.5, std::rand() / (double)RAND_MAX - 0.5);
        const std::vector<cd> y = inverse_dft_any(Y);
        CHECK((int)y.size() == T);
        double err = 0.0;
        for (int n = 0; n < T; n += (T > 2000 ? 61 : 1)) {
            cd sum = 0.0;
            for (int k = 0; k < T; ++k) {
                const long long q = ((long long)k * n) % T;
                sum += Y[k] * std::polar(1.0, 2.0 * M_PI * (double)q / T);
            }
            err = std::fmax(err, std::abs(sum / (double)T - y[n]));
        }
        CHECK(err < 1e-14);
    }
    std::printf("ok\n");
    return 0;
}
"""


def _run_program(tmp_path, name, program):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    lib = build.build()
    src = tmp_path / f"{name}.cu"
    src.write_text(program)
    exe = tmp_path / name
    csrc = os.path.join(ROOT, "paper_1710_08037_gb300", "csrc")
    subprocess.run([nvcc, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "include"), "-I", csrc,
                    str(src), "-o", str(exe), "-L", os.path.dirname(lib), "-lplv",
                    "-Xlinker", "-rpath", "-Xlinker", os.path.dirname(lib)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr


def test_tuner_work_lists(tmp_path):
    _run_program(tmp_path, "schedule_check", PROGRAM)


def test_any_length_plan_helpers(tmp_path):
    _run_program(tmp_path, "plan_check", PLAN_PROGRAM)
