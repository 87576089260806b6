// group.cuh -- internal: the grouped plan (plv_group) and the host-side
// layouts of its two work lists, shared by the plan builder (plv_api.cu) and
// the autotuner (tune.cu).  Not part of the public ABI.
#pragma once

#include <map>
#include <string>
#include <vector>

#include "common.cuh"

namespace plv {

// Makes a device current for the scope and restores the caller's.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev)
            cudaSetDevice(prev);
    }
};

}  // namespace plv

struct plv_group {
    int device = 0;
    plv_precision prec = PLV_PREC_FP32;
    std::vector<plv_problem> host;   // validated problems (FP32 path)
    unsigned mask = 0;
    plv::TcProblem *probs = nullptr;  // device descriptors (split paths)
    int4 *items = nullptr;            // device launch list (tiles and split parts)
    int nprob = 0, nitems = 0;        // nitems: entries of the launch list
    int ntiles = 0;                   // the plan's tiles
    plv::TcSplit split;               // device split-K parts, slots and counters
    bool any_diag = false;
    std::vector<plv::TcProblem> dp_host;  // host copies of the descriptors
    std::vector<int4> items_host;         // the plan's (problem, epoch, I, J), longest first
    // analytic-signal plan (problems with an input x)
    bool has_k1 = false;
    plv_dtype k1_dtype = PLV_F32;
    plv::K1Desc *k1_descs = nullptr;  // device
    int2 *k1_items = nullptr;         // device
    plv::K1Group k1{};
    std::vector<plv::K1Desc> k1_host;  // host copies of the K1 descriptors
    plv::GroupConfig cfg;              // current launch configuration
    // work lists replaced by the autotuner, kept until the plan is destroyed
    // (CUDA graphs captured before tuning still launch on them)
    std::vector<void *> retired;
};

namespace plv {

// The (problem, row pair) items of a grouped K1 plan: by assigned thread
// class (cls[M], default conv_class(M)), then by decreasing M, then problem
// order.  Fills kg's begin / count / max_M (per_sm, descs and items are left
// to the caller).
void k1_layout(const std::vector<K1Desc> &descs, const std::map<int, int> &cls,
               std::vector<int2> &items, K1Group &kg);

// The order in which a persistent grid of G CTAs takes a longest-first work
// list (cost[i] = K blocks of entry i, non-increasing) under a schedule: a
// permutation of 0 .. cost.size() - 1.
std::vector<int64_t> gram_order(const std::vector<int> &cost, int schedule, int G,
                                int tile_cost);

// Split K: parts per tile (1: whole) for factor f over tiles of nkb[i] K
// blocks, `chunk` K blocks per summation chunk, a grid of G CTAs.
void split_plan(const std::vector<int> &nkb, int chunk, int G, int f, std::vector<int> &parts);
// K blocks [lo, hi) of part s of S of a tile of nkb K blocks (whole chunks).
void part_range(int nkb, int chunk, int S, int s, int &lo, int &hi);
constexpr int kMaxSplitFactor = 64;
constexpr int kMinPartKb = 64;            // parts of at least 2048 samples
constexpr int64_t kMaxSplitSlots = 8192;  // slots of 128 KB: 1 GiB

// A grouped Gram's launch list under a configuration: items in the kernel's
// format (problem, epoch, I | J << 16, 1 + part or 0) in the schedule's order,
// and the split parts with the chunk slots and counters they need.
struct GramList {
    std::vector<int4> items;
    std::vector<SplitPart> parts;
    int nslots = 0, ntiles = 0;
};
GramList gram_list(const std::vector<TcProblem> &dp, const std::vector<int4> &tiles, int chunk,
                   int num_sms, const GroupConfig &cfg);
// Whether `list` runs every K block of every tile exactly once.
bool covers(const std::vector<TcProblem> &dp, const std::vector<int4> &tiles,
            const GramList &list);
// Device copies of a launch list; on success the caller owns *items and the
// pointers of *split.
plv_status upload_list(const GramList &list, cudaStream_t s, int4 **items, TcSplit *split);
void free_list(int4 *items, const TcSplit &split);

// The persistent grid of the grouped Gram launch for n tiles.
inline int gram_group_grid(const Handle &h, int n) { return n < h.num_sms ? n : h.num_sms; }

}  // namespace plv
