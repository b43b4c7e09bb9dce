// Host side of the multi-solve engine (include/lbm.h, "engine" section):
// a device arena with first-fit allocation (admission by footprint), slots
// that can be added and removed between chunks, per-velocity-set work lists
// (bundles of channels small enough to run a whole chunk in shared memory,
// tiles of the others), CUDA-graph capture of a chunk of time steps plus the
// per-solve reductions, and an autotuner of each velocity set's tile shape,
// cells per tile and tiles per grab and of the persistent grid.  Storage fp64 (fp64 arithmetic), fp32, fp16 or bf16
// (fp32 arithmetic); the device slot records are EngineSolve<double> for fp64
// and EngineSolve<float> otherwise.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <queue>
#include <vector>

#include "engine_launch.cuh"
#include "lbm.h"
#include "lbm_internal.h"

namespace lbm {
cudaError_t engine_step_fp32(int set_id, int N, const EngineLaunch& L, cudaStream_t st);
cudaError_t engine_step_half(int set_id, int N, const EngineLaunch& L, cudaStream_t st);
cudaError_t engine_step_bf16(int set_id, int N, const EngineLaunch& L, cudaStream_t st);
cudaError_t engine_step_fp64(int set_id, int N, const EngineLaunch& L, cudaStream_t st);
int engine_occupancy_fp32(int set_id, int N);
int engine_occupancy_half(int set_id, int N);
int engine_occupancy_bf16(int set_id, int N);
int engine_occupancy_fp64(int set_id, int N);
cudaError_t engine_resident_fp32(int set_id, int N, const ResidentLaunch& L, cudaStream_t st);
cudaError_t engine_resident_half(int set_id, int N, const ResidentLaunch& L, cudaStream_t st);
cudaError_t engine_resident_bf16(int set_id, int N, const ResidentLaunch& L, cudaStream_t st);
cudaError_t engine_resident_fp64(int set_id, int N, const ResidentLaunch& L, cudaStream_t st);
int engine_resident_attr_fp32(int set_id, int N, size_t smem);
int engine_resident_attr_half(int set_id, int N, size_t smem);
int engine_resident_attr_bf16(int set_id, int N, size_t smem);
int engine_resident_attr_fp64(int set_id, int N, size_t smem);
cudaError_t engine_reduce(const void* solves, const int* active, double* out, int nslots,
                          cudaStream_t st);
cudaError_t engine_reduce_fp64(const void* solves, const int* active, double* out, int nslots,
                               cudaStream_t st);
cudaError_t engine_advance(unsigned int* seed, unsigned int by, cudaStream_t st);
}  // namespace lbm

namespace {

constexpr int kGroups = 18;        // 6 compiled velocity sets x Hermite orders 2..4
constexpr int kMaxChunk = 1000;    // steps per captured chunk
constexpr int kLanes = 4;          // concurrent streams inside a captured chunk

size_t al256(size_t n) { return (n + 255) & ~size_t(255); }

// First-fit allocator over [0, size) with 256-byte granularity.
class Arena {
  public:
    void reset(size_t size) {
        free_.clear();
        if (size) free_[0] = size;
    }
    bool alloc(size_t n, size_t& off) {
        n = al256(n);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            off = it->first;
            const size_t rest = it->second - n, o2 = it->first + n;
            free_.erase(it);
            if (rest) free_[o2] = rest;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t n) {
        n = al256(n);
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t largest() const {
        size_t m = 0;
        for (const auto& kv : free_) m = std::max(m, kv.second);
        return m;
    }

  private:
    std::map<size_t, size_t> free_;
};

struct SlotLayout {
    size_t f0, f1, rho, ux, uy, prev, total;
};

SlotLayout slot_layout(int V, size_t ncell, size_t elem) {
    SlotLayout L{};
    size_t off = 0;
    auto take = [&](size_t n) { size_t o = off; off = al256(off + n); return o; };
    L.f0 = take(size_t(V) * ncell * elem);
    L.f1 = take(size_t(V) * ncell * elem);
    L.rho = take(ncell * 8);
    L.ux = take(ncell * 8);
    L.uy = take(ncell * 8);
    L.prev = take(ncell * 8);
    L.total = off;
    return L;
}

struct GroupWork {
    int g;
    bool tiled, res;       // the group has tiles / bundles
    int grid, rgrid;       // persistent grids (set at capture)
    bool operator==(const GroupWork& o) const { return g == o.g && tiled == o.tiled && res == o.res; }
};

struct EngSlot {
    bool used = false;
    lbm::SolveSpec spec;
    size_t off = 0, bytes = 0;
    long steps = 0;
    int group = -1;
    // device buffers of the solve (also in its device record)
    void* f[2] = {nullptr, nullptr};
    double *rho = nullptr, *ux = nullptr, *uy = nullptr, *prev = nullptr;
    unsigned* status = nullptr;
    int phase = 0;
    double tau = 0, g = 0;
};

__global__ void k_fill_ones(double* p, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = 1.0;
}

int cuda_rc(cudaError_t e) {
    return e == cudaSuccess ? LBM_OK : (e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA);
}

}  // namespace

struct lbm_engine {
    int precision = LBM_FP32;
    cudaStream_t stream = nullptr;
    bool own_stream = false, own_arena = false;
    char* base = nullptr;
    size_t bytes = 0, ctrl = 0;
    Arena arena;                               // over [ctrl, bytes)
    int max_slots = 0;
    size_t tile_cap = 0;
    void* d_solves = nullptr;                  // EngineSolve<double or float>[max_slots]
    size_t rec_bytes = 0;                      // bytes of one record
    int* d_active = nullptr;
    double* d_results = nullptr;
    unsigned* d_status = nullptr;
    int* d_ntiles = nullptr;
    int* d_counters = nullptr;
    unsigned* d_seed = nullptr;
    lbm::EngineTile* d_tiles = nullptr;
    std::vector<EngSlot> slots;
    std::vector<unsigned char> h_rec;          // host copies of the records
    std::vector<int> h_active;
    std::vector<double> h_results;
    // asynchronous chunks: per outstanding launch, its results copied in
    // stream order into pinned host memory, and an event marking the copy
    double* pinned = nullptr;                  // 2 x 4 x max_slots doubles
    cudaEvent_t ev_done[2] = {};
    int pending = 0, head = 0;                 // outstanding launches, oldest one
    int K = 100;
    double bps_factor = 1.0;   // fraction of the occupancy limit used for the grid
    // schedule of each group's tiled launches
    int grab[kGroups];         // tiles taken per atomic grab
    int tile_tws[kGroups];     // tile width 2^tws columns (0: linear tiles)
    int tile_m[kGroups];       // tiles of tile_m x 128 nodes
    int sms = 0;
    bool tiles_dirty = true, graph_dirty = true;
    // resident chunks
    bool resident = true;
    size_t res_smem = 0;                       // dynamic shared memory per resident block
    int res_occ[kGroups];                      // resident blocks per SM, -1: not yet queried
    lbm::ResBundle* d_bundles = nullptr;       // max_slots entries
    lbm::ResChannel* d_chans = nullptr;        // max_slots entries
    int* d_nbundles = nullptr;                 // per group: counts, then offsets
    int* d_rcounters = nullptr;                // per group
    cudaStream_t side[kLanes - 1] = {};        // forks of the chunk graph
    cudaEvent_t ev_fork = nullptr, ev_join[kLanes - 1] = {};
    std::vector<GroupWork> plan;               // present groups and their work
    int n_tiled = 0, n_resident = 0;          // solves per path at the last rebuild
    cudaGraphExec_t exec = nullptr;
};

namespace {

int group_of(const lbm::SolveSpec& s) { return s.set_id * 3 + (s.N - 2); }

bool is16(int p) { return p == LBM_FP16 || p == LBM_BF16; }

int occupancy(const lbm_engine* e, int group) {
    const int set = group / 3, N = group % 3 + 2;
    const int b = e->precision == LBM_FP16   ? lbm::engine_occupancy_half(set, N)
                  : e->precision == LBM_BF16 ? lbm::engine_occupancy_bf16(set, N)
                  : e->precision == LBM_FP64 ? lbm::engine_occupancy_fp64(set, N)
                                             : lbm::engine_occupancy_fp32(set, N);
    return std::max(1, b);
}

// resident blocks per SM of the group's resident kernel at res_smem (0: unusable)
int res_occupancy(lbm_engine* e, int group) {
    if (e->res_occ[group] < 0) {
        const int set = group / 3, N = group % 3 + 2;
        e->res_occ[group] =
            e->precision == LBM_FP16   ? lbm::engine_resident_attr_half(set, N, e->res_smem)
            : e->precision == LBM_BF16 ? lbm::engine_resident_attr_bf16(set, N, e->res_smem)
            : e->precision == LBM_FP64 ? lbm::engine_resident_attr_fp64(set, N, e->res_smem)
                                       : lbm::engine_resident_attr_fp32(set, N, e->res_smem);
    }
    return e->res_occ[group];
}

// shared-memory footprint of a channel in a bundle: V planes of Nx (Ny + 2 maxey)
size_t res_bytes(const lbm::SolveSpec& s) {
    return size_t(s.V) * s.Nx * (s.Ny + 2 * s.maxey) * s.elem;
}

bool res_eligible(lbm_engine* e, const EngSlot& sl) {
    const size_t n = size_t(sl.spec.Nx) * sl.spec.Ny;
    return e->resident && res_bytes(sl.spec) <= e->res_smem &&
           ((n + 31) & ~size_t(31)) <= size_t(lbm::kResNodes) && res_occupancy(e, sl.group) > 0;
}

struct Bin {
    size_t bytes = 0;
    int nodes = 0;
    std::vector<int> members;
};

struct ResItem {
    size_t bytes;
    int nodes;     // padded to 32
    int slot;
};

// Pack resident channels into bundles for `grid` persistent blocks: the
// fewest whole waves (bundles = waves x grid) whose bundles respect the
// shared-memory, node and channel limits, the channels placed largest first
// on the least-loaded bundle (by nodes), so that every block gets about the
// same work.  Bundles are returned largest first (the blocks take them in
// that order).
std::vector<Bin> pack_bundles(std::vector<ResItem> items, size_t capb, int grid) {
    std::vector<Bin> out;
    if (items.empty()) return out;
    std::stable_sort(items.begin(), items.end(),
                     [](const ResItem& a, const ResItem& b) { return a.nodes > b.nodes; });
    size_t total_b = 0, total_n = 0;
    for (const ResItem& it : items) {
        total_b += it.bytes;
        total_n += size_t(it.nodes);
    }
    const size_t per_wave_b = capb * size_t(grid), per_wave_n = size_t(lbm::kResNodes) * grid;
    size_t waves = std::max<size_t>(1, std::max((total_b + per_wave_b - 1) / per_wave_b,
                                                (total_n + per_wave_n - 1) / per_wave_n));
    using Load = std::pair<long long, int>;   // (nodes, bundle)
    for (;; ++waves) {
        const size_t nb = std::min(items.size(), waves * size_t(grid));
        std::vector<Bin> bins(nb);
        std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
        for (size_t i = 0; i < nb; ++i) heap.push({0, int(i)});
        std::vector<Load> skipped;
        bool ok = true;
        for (const ResItem& it : items) {
            bool placed = false;
            skipped.clear();
            while (!heap.empty()) {
                const Load top = heap.top();
                heap.pop();
                Bin& b = bins[top.second];
                if (b.bytes + it.bytes <= capb && b.nodes + it.nodes <= lbm::kResNodes &&
                    int(b.members.size()) < lbm::kResMaxCh) {
                    b.bytes += it.bytes;
                    b.nodes += it.nodes;
                    b.members.push_back(it.slot);
                    heap.push({b.nodes, top.second});
                    placed = true;
                    break;
                }
                skipped.push_back(top);
            }
            for (const Load& l : skipped) heap.push(l);
            if (!placed) {
                ok = false;
                break;
            }
        }
        if (!ok) continue;
        for (Bin& b : bins)
            if (!b.members.empty()) out.push_back(std::move(b));
        std::stable_sort(out.begin(), out.end(),
                         [](const Bin& a, const Bin& b) { return a.nodes > b.nodes; });
        return out;
    }
}

// Work lists: per group, bundles of resident channels (pack_bundles) and
// tiles of the others.
int rebuild_tiles(lbm_engine* e) {
    std::vector<lbm::EngineTile> t;
    std::vector<lbm::ResBundle> bundles;
    std::vector<lbm::ResChannel> chans;
    std::vector<GroupWork> plan;
    std::vector<int> counts(2 * kGroups, 0), nbund(2 * kGroups, 0);   // count, offset
    for (int g = 0; g < kGroups; ++g) {
        const size_t start = t.size(), bstart = bundles.size();
        std::vector<int> res;
        for (int s = 0; s < e->max_slots; ++s) {
            const EngSlot& sl = e->slots[s];
            if (!sl.used || sl.group != g) continue;
            if (res_eligible(e, sl)) {
                res.push_back(s);
                continue;
            }
            const int Nx = sl.spec.Nx, Ny = sl.spec.Ny, cells = e->tile_m[g] * lbm::kBlock;
            const int tw = e->tile_tws[g] ? 1 << e->tile_tws[g] : 0, th = tw ? cells / tw : 0;
            if (tw && Nx % tw == 0 && Ny >= th) {
                // at most 2 Nx Ny / cells tiles (Ny >= th)
                for (int y0 = 0; y0 < Ny; y0 += th)
                    for (int x0 = 0; x0 < Nx; x0 += tw)
                        t.push_back({s, y0 * Nx + x0, e->tile_tws[g]});
            } else {
                for (int c0 = 0; c0 < Nx * Ny; c0 += cells)
                    t.push_back({s, c0, 0});
            }
        }
        std::vector<ResItem> items;
        for (int s : res)
            items.push_back({res_bytes(e->slots[s].spec),
                             (e->slots[s].spec.Nx * e->slots[s].spec.Ny + 31) & ~31, s});
        const int rgrid = res.empty() ? 1 : std::max(1, res_occupancy(e, g)) * e->sms;
        const std::vector<Bin> bins = pack_bundles(std::move(items), e->res_smem, rgrid);
        for (const Bin& b : bins) {
            lbm::ResBundle rb{int(chans.size()), int(b.members.size()), 0, 0};
            int off = 0;
            for (int s : b.members) {
                const lbm::SolveSpec& sp = e->slots[s].spec;
                const int n = sp.Nx * sp.Ny;
                chans.push_back({s, rb.nodes, off, n});
                rb.nodes += (n + 31) & ~31;
                off += int(res_bytes(sp) / sp.elem);
            }
            bundles.push_back(rb);
        }
        counts[g] = int(t.size() - start);
        counts[kGroups + g] = int(start);
        nbund[g] = int(bundles.size() - bstart);
        nbund[kGroups + g] = int(bstart);
        if (counts[g] || nbund[g]) plan.push_back({g, counts[g] > 0, nbund[g] > 0, 0, 0});
    }
    if (t.size() > e->tile_cap || bundles.size() > size_t(e->max_slots)) return LBM_ENOMEM;
    cudaError_t err = cudaSuccess;
    if (!t.empty())
        err = cudaMemcpyAsync(e->d_tiles, t.data(), t.size() * sizeof(lbm::EngineTile),
                              cudaMemcpyHostToDevice, e->stream);
    if (err == cudaSuccess && !bundles.empty())
        err = cudaMemcpyAsync(e->d_bundles, bundles.data(), bundles.size() * sizeof(lbm::ResBundle),
                              cudaMemcpyHostToDevice, e->stream);
    if (err == cudaSuccess && !chans.empty())
        err = cudaMemcpyAsync(e->d_chans, chans.data(), chans.size() * sizeof(lbm::ResChannel),
                              cudaMemcpyHostToDevice, e->stream);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(e->d_ntiles, counts.data(), 2 * kGroups * sizeof(int),
                              cudaMemcpyHostToDevice, e->stream);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(e->d_nbundles, nbund.data(), 2 * kGroups * sizeof(int),
                              cudaMemcpyHostToDevice, e->stream);

    if (err != cudaSuccess) return cuda_rc(err);
    e->n_resident = int(chans.size());
    e->n_tiled = 0;
    for (const EngSlot& sl : e->slots) e->n_tiled += sl.used;
    e->n_tiled -= e->n_resident;
    // the graph reads counts and offsets from device memory: only a change of
    // the launches themselves needs a new capture
    if (!(plan == e->plan)) {
        e->graph_dirty = true;
        e->plan = plan;
    }
    e->tiles_dirty = false;
    return LBM_OK;
}

// One chunk of K steps + the reductions + the seed advance, on the stream.
// Independent work items run on forks of the stream inside the captured
// chunk: the resident bundles of all groups (K steps per launch) and the K
// per-step launches of each group's tiles.  The items touch disjoint solves,
// so they overlap on the GPU and one group's kernel tail is filled by
// another's blocks.  Items are dealt to kLanes streams in order.
int enqueue_chunk(lbm_engine* e) {
    bool any_t = false, any_r = false;
    int items = 0;
    for (const GroupWork& w : e->plan) {
        any_t |= w.tiled;
        any_r |= w.res;
        items += w.tiled;
    }
    items += any_r;
    cudaError_t err = cudaSuccess;
    if (any_t) err = cudaMemsetAsync(e->d_counters, 0, sizeof(int) * kGroups * e->K, e->stream);
    if (any_r && err == cudaSuccess)
        err = cudaMemsetAsync(e->d_rcounters, 0, sizeof(int) * kGroups, e->stream);
    if (err != cudaSuccess) return cuda_rc(err);
    const int lanes = std::min(items, kLanes);
    auto lane = [&](int item) { return item % kLanes == 0 ? e->stream : e->side[item % kLanes - 1]; };
    if (lanes > 1) {
        err = cudaEventRecord(e->ev_fork, e->stream);
        for (int l = 1; l < lanes && err == cudaSuccess; ++l)
            err = cudaStreamWaitEvent(e->side[l - 1], e->ev_fork, 0);
        if (err != cudaSuccess) return cuda_rc(err);
    }
    int item = 0;
    if (any_r) {
        const cudaStream_t rs = lane(item++);
        for (const GroupWork& w : e->plan) {
            if (!w.res) continue;
            lbm::ResidentLaunch L{};
            L.solves = e->d_solves;
            L.bundles = e->d_bundles;
            L.chans = e->d_chans;
            L.nbundles = e->d_nbundles + w.g;
            L.bundle_off = e->d_nbundles + kGroups + w.g;
            L.counter = e->d_rcounters + w.g;
            L.seed = e->d_seed;
            L.K = e->K;
            L.grid = w.rgrid;
            L.smem = e->res_smem;
            const int set = w.g / 3, N = w.g % 3 + 2;
            err = e->precision == LBM_FP16   ? lbm::engine_resident_half(set, N, L, rs)
                  : e->precision == LBM_BF16 ? lbm::engine_resident_bf16(set, N, L, rs)
                  : e->precision == LBM_FP64 ? lbm::engine_resident_fp64(set, N, L, rs)
                                             : lbm::engine_resident_fp32(set, N, L, rs);
            if (err != cudaSuccess) return cuda_rc(err);
        }
    }
    for (const GroupWork& w : e->plan) {
        if (!w.tiled) continue;
        const cudaStream_t ts = lane(item++);
        for (int i = 0; i < e->K; ++i) {
            lbm::EngineLaunch L{};
            L.solves = e->d_solves;
            L.tiles = e->d_tiles;
            L.ntiles = e->d_ntiles + w.g;
            L.tile_off = e->d_ntiles + kGroups + w.g;
            L.counter = e->d_counters + i * kGroups + w.g;
            L.seed = e->d_seed;
            L.parity = i & 1;
            L.emit = i == e->K - 1 ? 1 : (i == e->K - 2 ? 2 : 0);
            L.chunk = e->grab[w.g];
            L.lm = e->tile_m[w.g] == 4 ? 2 : e->tile_m[w.g] - 1;
            L.grid = w.grid;
            const int set = w.g / 3, N = w.g % 3 + 2;
            err = e->precision == LBM_FP16   ? lbm::engine_step_half(set, N, L, ts)
                  : e->precision == LBM_BF16 ? lbm::engine_step_bf16(set, N, L, ts)
                  : e->precision == LBM_FP64 ? lbm::engine_step_fp64(set, N, L, ts)
                                             : lbm::engine_step_fp32(set, N, L, ts);
            if (err != cudaSuccess) return cuda_rc(err);
        }
    }
    for (int l = 1; l < lanes; ++l) {
        err = cudaEventRecord(e->ev_join[l - 1], e->side[l - 1]);
        if (err == cudaSuccess) err = cudaStreamWaitEvent(e->stream, e->ev_join[l - 1], 0);
        if (err != cudaSuccess) return cuda_rc(err);
    }
    err = e->precision == LBM_FP64
              ? lbm::engine_reduce_fp64(e->d_solves, e->d_active, e->d_results, e->max_slots, e->stream)
              : lbm::engine_reduce(e->d_solves, e->d_active, e->d_results, e->max_slots, e->stream);
    if (err == cudaSuccess) err = lbm::engine_advance(e->d_seed, unsigned(e->K), e->stream);
    return cuda_rc(err);
}

int recapture(lbm_engine* e) {
    for (GroupWork& w : e->plan) {
        w.grid = std::max(1, int(std::lround(occupancy(e, w.g) * e->bps_factor))) * e->sms;
        w.rgrid = w.res ? std::max(1, res_occupancy(e, w.g)) * e->sms : 0;
    }
    if (e->exec) {
        cudaGraphExecDestroy(e->exec);
        e->exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    cudaError_t err = cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal);
    if (err != cudaSuccess) return cuda_rc(err);
    const int rc = enqueue_chunk(e);
    err = cudaStreamEndCapture(e->stream, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (err != cudaSuccess) return cuda_rc(err);
    err = cudaGraphInstantiate(&e->exec, g, 0);
    cudaGraphDestroy(g);
    if (err != cudaSuccess) return cuda_rc(err);
    e->graph_dirty = false;
    return LBM_OK;
}

int prepare(lbm_engine* e) {
    if (e->tiles_dirty) {
        const int rc = rebuild_tiles(e);
        if (rc) return rc;
    }
    if (e->graph_dirty && !e->plan.empty()) return recapture(e);
    return LBM_OK;
}

int fetch_results(lbm_engine* e, double* out) {
    cudaError_t err = cudaMemcpyAsync(e->h_results.data(), e->d_results,
                                      sizeof(double) * 4 * e->max_slots, cudaMemcpyDeviceToHost,
                                      e->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(e->stream);
    if (err != cudaSuccess) return cuda_rc(err);
    if (out) std::memcpy(out, e->h_results.data(), sizeof(double) * 4 * e->max_slots);
    return LBM_OK;
}

// Device record of a slot (compute type C), its initial state fbar = rho w,
// first relaxation and moments (the single-solve init kernel).
template <typename C>
cudaError_t upload_and_init(lbm_engine* e, int slot, double Kn, const double* rho_host) {
    const EngSlot& sl = e->slots[slot];
    const lbm::SolveSpec& spec = sl.spec;
    auto& h = *reinterpret_cast<lbm::EngineSolve<C>*>(e->h_rec.data() + size_t(slot) * e->rec_bytes);
    std::memset(&h, 0, sizeof(h));
    lbm::fill_params(spec, h.k);
    h.f[0] = sl.f[0];
    h.f[1] = sl.f[1];
    h.rho = sl.rho;
    h.ux = sl.ux;
    h.uy = sl.uy;
    h.prev = sl.prev;
    h.status = sl.status;
    h.phase = sl.phase;
    h.kn = Kn;
    h.tau = sl.tau;
    h.g = sl.g;
    lbm::DevBufs db{};
    db.f[0] = h.f[0];
    db.f[1] = h.f[1];
    db.rho = h.rho;
    db.ux = h.ux;
    db.uy = h.uy;
    db.prev_ux = h.prev;
    db.status = h.status;
    const int n = spec.Nx * spec.Ny;
    cudaError_t err = cudaMemcpyAsync(static_cast<char*>(e->d_solves) + size_t(slot) * e->rec_bytes,
                                      &h, sizeof(h), cudaMemcpyHostToDevice, e->stream);
    if (err == cudaSuccess) err = cudaMemsetAsync(h.status, 0, sizeof(unsigned), e->stream);
    if (err == cudaSuccess) {
        if (rho_host) {
            err = cudaMemcpyAsync(h.prev, rho_host, size_t(n) * 8, cudaMemcpyHostToDevice, e->stream);
        } else {
            k_fill_ones<<<(n + 255) / 256, 256, 0, e->stream>>>(h.prev, n);
            err = cudaGetLastError();
        }
    }
    if (err == cudaSuccess) {
        lbm::KParams<C> k = h.k;
        k.emit = 1;
        k.seed = 0u;
        if constexpr (sizeof(C) == 8)
            err = lbm::launch_init_fp64(k, spec.N, h.prev, h.f[0], db, e->stream);
        else
            err = is16(e->precision)
                      ? lbm::launch_init_fp16(k, spec.N, e->precision == LBM_BF16, h.prev, h.f[0], db,
                                              e->stream)
                      : lbm::launch_init_fp32(k, spec.N, h.prev, h.f[0], db, e->stream);
    }
    return err;
}

}  // namespace

extern "C" {

int lbm_engine_solve_bytes(const lbm_dvm* dvm, int Nx, int Ny, int precision, size_t* bytes) {
    if (!dvm || !bytes || Nx < 1 || Ny < 1 || dvm->V < 1 || dvm->V > LBM_MAX_V) return LBM_EINVAL;
    if (precision != LBM_FP32 && precision != LBM_FP64 && !is16(precision)) return LBM_EINVAL;
    *bytes = slot_layout(dvm->V, size_t(Nx) * Ny, lbm::elem_bytes(precision)).total;
    return LBM_OK;
}

int lbm_engine_create(int precision, int max_solves, void* arena, size_t arena_bytes, void* stream,
                      lbm_engine** out) {
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    if ((precision != LBM_FP32 && precision != LBM_FP64 && !is16(precision)) || max_solves < 1 ||
        max_solves > 65536)
        return LBM_EINVAL;
    if (arena && (reinterpret_cast<uintptr_t>(arena) & 255)) return LBM_EINVAL;
    lbm_engine* e = new (std::nothrow) lbm_engine();
    if (!e) return LBM_ENOMEM;
    e->precision = precision;
    e->max_slots = max_solves;
    const size_t elem = lbm::elem_bytes(precision);
    // tiles: at most two per 128 nodes of the smallest lattice that fits (2-D
    // tiles clipped at the top row), plus a partial tile per solve
    const size_t max_cells = arena_bytes / (2 * 16 * elem);
    e->tile_cap = 2 * (max_cells / lbm::kBlock) + size_t(max_solves) + 1;
    size_t off = 0;
    auto take = [&](size_t n) { size_t o = off; off = al256(off + n); return o; };
    e->rec_bytes = precision == LBM_FP64 ? sizeof(lbm::EngineSolve<double>)
                                         : sizeof(lbm::EngineSolve<float>);
    const size_t o_solves = take(e->rec_bytes * max_solves);
    const size_t o_active = take(sizeof(int) * max_solves);
    const size_t o_results = take(sizeof(double) * 4 * max_solves);
    const size_t o_status = take(sizeof(unsigned) * max_solves);
    const size_t o_ntiles = take(sizeof(int) * 2 * kGroups);
    const size_t o_nbundles = take(sizeof(int) * 2 * kGroups);
    const size_t o_rcounters = take(sizeof(int) * kGroups);
    const size_t o_bundles = take(sizeof(lbm::ResBundle) * max_solves);
    const size_t o_chans = take(sizeof(lbm::ResChannel) * max_solves);
    const size_t o_counters = take(sizeof(int) * kGroups * kMaxChunk);
    const size_t o_seed = take(sizeof(unsigned));
    const size_t o_tiles = take(sizeof(lbm::EngineTile) * e->tile_cap);
    e->ctrl = off;
    if (arena_bytes <= e->ctrl) { delete e; return LBM_ENOMEM; }
    if (arena) {
        e->base = static_cast<char*>(arena);
    } else {
        if (cudaMalloc(&e->base, arena_bytes) != cudaSuccess) { delete e; return LBM_ENOMEM; }
        e->own_arena = true;
    }
    e->bytes = arena_bytes;
    e->arena.reset(arena_bytes - e->ctrl);
    e->d_solves = e->base + o_solves;
    e->d_active = reinterpret_cast<int*>(e->base + o_active);
    e->d_results = reinterpret_cast<double*>(e->base + o_results);
    e->d_status = reinterpret_cast<unsigned*>(e->base + o_status);
    e->d_ntiles = reinterpret_cast<int*>(e->base + o_ntiles);
    e->d_nbundles = reinterpret_cast<int*>(e->base + o_nbundles);
    e->d_rcounters = reinterpret_cast<int*>(e->base + o_rcounters);
    e->d_bundles = reinterpret_cast<lbm::ResBundle*>(e->base + o_bundles);
    e->d_chans = reinterpret_cast<lbm::ResChannel*>(e->base + o_chans);
    for (int g = 0; g < kGroups; ++g) {
        e->res_occ[g] = -1;
        e->grab[g] = 4;
        e->tile_tws[g] = 0;
        e->tile_m[g] = 1;
    }
    e->d_counters = reinterpret_cast<int*>(e->base + o_counters);
    e->d_seed = reinterpret_cast<unsigned*>(e->base + o_seed);
    e->d_tiles = reinterpret_cast<lbm::EngineTile*>(e->base + o_tiles);
    e->slots.resize(max_solves);
    e->h_rec.assign(e->rec_bytes * size_t(max_solves), 0);
    e->h_active.assign(max_solves, 0);
    e->h_results.assign(4 * size_t(max_solves), 0.0);
    if (cudaMallocHost(&e->pinned, sizeof(double) * 8 * size_t(max_solves)) != cudaSuccess) {
        cudaGetLastError();
        lbm_engine_destroy(e);
        return LBM_ENOMEM;
    }
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&e->sms, cudaDevAttrMultiProcessorCount, dev);
    int optin = 0;
    if (err == cudaSuccess)
        err = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // the resident kernels' static shared memory is under 2 KiB
    e->res_smem = optin > 4096 ? size_t(optin - 4096) & ~size_t(255) : 0;
    for (int l = 0; l < kLanes - 1 && err == cudaSuccess; ++l) {
        err = cudaStreamCreateWithFlags(&e->side[l], cudaStreamNonBlocking);
        if (err == cudaSuccess) err = cudaEventCreateWithFlags(&e->ev_join[l], cudaEventDisableTiming);
    }
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&e->ev_fork, cudaEventDisableTiming);
    for (int l = 0; l < 2 && err == cudaSuccess; ++l)
        err = cudaEventCreateWithFlags(&e->ev_done[l], cudaEventDisableTiming);
    if (err == cudaSuccess) {
        if (stream) {
            e->stream = static_cast<cudaStream_t>(stream);
        } else {
            err = cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking);
            e->own_stream = err == cudaSuccess;
        }
    }
    if (err == cudaSuccess) err = cudaMemsetAsync(e->base, 0, e->ctrl, e->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(e->stream);
    if (err != cudaSuccess) {
        lbm_engine_destroy(e);
        return cuda_rc(err);
    }
    *out = e;
    return LBM_OK;
}

void lbm_engine_destroy(lbm_engine* e) {
    if (!e) return;
    if (e->stream) cudaStreamSynchronize(e->stream);
    if (e->exec) cudaGraphExecDestroy(e->exec);
    if (e->ev_fork) cudaEventDestroy(e->ev_fork);
    for (int l = 0; l < 2; ++l)
        if (e->ev_done[l]) cudaEventDestroy(e->ev_done[l]);
    if (e->pinned) cudaFreeHost(e->pinned);
    for (int l = 0; l < kLanes - 1; ++l) {
        if (e->ev_join[l]) cudaEventDestroy(e->ev_join[l]);
        if (e->side[l]) cudaStreamDestroy(e->side[l]);
    }
    if (e->own_arena && e->base) cudaFree(e->base);
    if (e->own_stream && e->stream) cudaStreamDestroy(e->stream);
    delete e;
}

int lbm_engine_add(lbm_engine* e, const lbm_dvm* dvm, int order, int Nx, int Ny, double Kn,
                   double force, const double* rho_host, int* slot_out) {
    if (!e || !slot_out) return LBM_EINVAL;
    lbm::SolveSpec spec;
    int rc = lbm::prepare_spec(dvm, order, Nx, Ny, Kn, force, e->precision, spec);
    if (rc) return rc;
    if (spec.set_id < 0) return LBM_ENOTSUP;       // only compiled velocity sets
    int slot = -1;
    for (int s = 0; s < e->max_slots; ++s)
        if (!e->slots[s].used) { slot = s; break; }
    if (slot < 0) return LBM_ENOMEM;
    const SlotLayout L = slot_layout(spec.V, size_t(Nx) * Ny, spec.elem);
    size_t off = 0;
    if (!e->arena.alloc(L.total, off)) return LBM_ENOMEM;
    char* b = e->base + e->ctrl + off;
    EngSlot& sl = e->slots[slot];
    sl.used = true;
    sl.spec = spec;
    sl.off = off;
    sl.bytes = L.total;
    sl.steps = 0;
    sl.group = group_of(spec);
    sl.f[0] = b + L.f0;
    sl.f[1] = b + L.f1;
    sl.rho = reinterpret_cast<double*>(b + L.rho);
    sl.ux = reinterpret_cast<double*>(b + L.ux);
    sl.uy = reinterpret_cast<double*>(b + L.uy);
    sl.prev = reinterpret_cast<double*>(b + L.prev);
    sl.status = e->d_status + slot;
    sl.phase = 0;
    sl.tau = spec.tau;
    sl.g = force;
    cudaError_t err = e->precision == LBM_FP64 ? upload_and_init<double>(e, slot, Kn, rho_host)
                                               : upload_and_init<float>(e, slot, Kn, rho_host);
    e->h_active[slot] = 1;
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(e->d_active + slot, &e->h_active[slot], sizeof(int),
                              cudaMemcpyHostToDevice, e->stream);
    if (err != cudaSuccess) {
        e->h_active[slot] = 0;
        sl.used = false;
        e->arena.release(off, L.total);
        return cuda_rc(err);
    }
    e->tiles_dirty = true;
    *slot_out = slot;
    return LBM_OK;
}

int lbm_engine_remove(lbm_engine* e, int slot) {
    if (!e || slot < 0 || slot >= e->max_slots || !e->slots[slot].used) return LBM_EINVAL;
    EngSlot& sl = e->slots[slot];
    e->h_active[slot] = 0;
    // stream-ordered: work already queued for this slot finishes before any
    // later use of its memory (a new solve's set-up goes on the same stream)
    cudaError_t err = cudaMemcpyAsync(e->d_active + slot, &e->h_active[slot], sizeof(int),
                                      cudaMemcpyHostToDevice, e->stream);
    if (err != cudaSuccess) return cuda_rc(err);
    e->arena.release(sl.off, sl.bytes);
    sl.used = false;
    e->tiles_dirty = true;
    return LBM_OK;
}

int lbm_engine_set_resident(lbm_engine* e, int enable) {
    if (!e || (enable != 0 && enable != 1)) return LBM_EINVAL;
    if (e->resident != (enable == 1)) {
        e->resident = enable == 1;
        e->tiles_dirty = true;
    }
    return LBM_OK;
}

int lbm_engine_paths(lbm_engine* e, int* tiled, int* resident) {
    if (!e) return LBM_EINVAL;
    const int rc = prepare(e);
    if (rc) return rc;
    if (tiled) *tiled = e->n_tiled;
    if (resident) *resident = e->n_resident;
    return LBM_OK;
}

int lbm_engine_set_chunk(lbm_engine* e, int steps) {
    if (!e || steps < 2 || steps > kMaxChunk || (steps & 1)) return LBM_EINVAL;
    if (steps != e->K) {
        e->K = steps;
        e->graph_dirty = true;
    }
    return LBM_OK;
}

int lbm_engine_launch(lbm_engine* e, int chunks) {
    if (!e || chunks < 0 || e->pending >= 2) return LBM_EINVAL;
    int rc = prepare(e);
    if (rc) return rc;
    if (!e->plan.empty()) {
        for (int c = 0; c < chunks; ++c) {
            const cudaError_t err = cudaGraphLaunch(e->exec, e->stream);
            if (err != cudaSuccess) return cuda_rc(err);
        }
        for (auto& sl : e->slots)
            if (sl.used) sl.steps += long(chunks) * e->K;
    }
    const int b = (e->head + e->pending) & 1;
    cudaError_t err = cudaMemcpyAsync(e->pinned + size_t(b) * 4 * e->max_slots, e->d_results,
                                      sizeof(double) * 4 * e->max_slots, cudaMemcpyDeviceToHost,
                                      e->stream);
    if (err == cudaSuccess) err = cudaEventRecord(e->ev_done[b], e->stream);
    if (err != cudaSuccess) return cuda_rc(err);
    ++e->pending;
    return LBM_OK;
}

int lbm_engine_wait(lbm_engine* e, double* results) {
    if (!e || e->pending == 0) return LBM_EINVAL;
    const int b = e->head;
    const cudaError_t err = cudaEventSynchronize(e->ev_done[b]);
    if (err != cudaSuccess) return cuda_rc(err);
    if (results)
        std::memcpy(results, e->pinned + size_t(b) * 4 * e->max_slots,
                    sizeof(double) * 4 * e->max_slots);
    e->head ^= 1;
    --e->pending;
    return LBM_OK;
}

int lbm_engine_run(lbm_engine* e, int chunks, double* results) {
    if (!e || chunks < 0 || e->pending) return LBM_EINVAL;
    int rc = prepare(e);
    if (rc) return rc;
    if (!e->plan.empty()) {
        for (int c = 0; c < chunks; ++c) {
            const cudaError_t err = cudaGraphLaunch(e->exec, e->stream);
            if (err != cudaSuccess) return cuda_rc(err);
        }
        for (auto& sl : e->slots)
            if (sl.used) sl.steps += long(chunks) * e->K;
    }
    return fetch_results(e, results);
}

namespace {

// Time two chunks of the current schedule (after a warm-up chunk); the three
// chunks advance the solves and are counted.
int time_schedule(lbm_engine* e, cudaEvent_t a, cudaEvent_t b, float* ms) {
    int rc = prepare(e);
    if (rc) return rc;
    cudaGraphLaunch(e->exec, e->stream);      // warm-up chunk
    cudaEventRecord(a, e->stream);
    cudaGraphLaunch(e->exec, e->stream);
    cudaGraphLaunch(e->exec, e->stream);
    cudaEventRecord(b, e->stream);
    if (cudaEventSynchronize(b) != cudaSuccess) return LBM_ECUDA;
    cudaEventElapsedTime(ms, a, b);
    for (auto& sl : e->slots)
        if (sl.used) sl.steps += 3L * e->K;
    return LBM_OK;
}

}  // namespace

// Coordinate search over the tiled groups' schedules (groups run together in
// a chunk, so each candidate is timed on the whole chunk): one tile shape and
// cells per tile for all groups, then per group its own shape and its grab,
// last the grid fraction.
int lbm_engine_autotune(lbm_engine* e, double* best_ms_per_step) {
    if (!e || e->pending) return LBM_EINVAL;
    int rc = prepare(e);
    if (rc) return rc;
    if (e->plan.empty()) return LBM_OK;
    static const int shapes[][2] = {{0, 1}, {0, 2}, {0, 4}, {5, 1}, {5, 2}, {5, 4},
                                    {6, 1}, {6, 2}, {6, 4}, {7, 2}, {7, 4}};
    const int grabs[] = {1, 2, 4, 8, 16};
    std::vector<int> tiled;
    for (const GroupWork& w : e->plan)
        if (w.tiled) tiled.push_back(w.g);
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return LBM_ECUDA;
    if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return LBM_ECUDA; }
    float best = HUGE_VALF, ms = 0.f;
    // the current schedule first
    e->graph_dirty = true;
    rc = time_schedule(e, a, b, &best);
    // one shape for every tiled group
    if (!tiled.empty()) {
        const int tws0 = e->tile_tws[tiled[0]], m0 = e->tile_m[tiled[0]];
        int btws = tws0, bm = m0;
        for (const auto& sh : shapes) {
            if (rc) break;
            if (sh[0] == tws0 && sh[1] == m0) continue;
            for (int g : tiled) {
                e->tile_tws[g] = sh[0];
                e->tile_m[g] = sh[1];
            }
            e->tiles_dirty = e->graph_dirty = true;
            if ((rc = time_schedule(e, a, b, &ms))) break;
            if (ms < best) {
                best = ms;
                btws = sh[0];
                bm = sh[1];
            }
        }
        for (int g : tiled) {
            e->tile_tws[g] = btws;
            e->tile_m[g] = bm;
        }
        e->tiles_dirty = e->graph_dirty = true;
    }
    // then each group's own shape and grab, a change kept only if it saves
    // more than 0.5 % (the timing noise of two chunks)
    for (int g : tiled) {
        const int tws0 = e->tile_tws[g], m0 = e->tile_m[g];   // timed already
        int btws = tws0, bm = m0;
        for (const auto& sh : shapes) {
            if (rc) break;
            if (sh[0] == tws0 && sh[1] == m0) continue;
            const int otws = e->tile_tws[g], om = e->tile_m[g];
            e->tile_tws[g] = sh[0];
            e->tile_m[g] = sh[1];
            e->tiles_dirty = e->graph_dirty = true;
            if ((rc = time_schedule(e, a, b, &ms))) break;
            if (ms < 0.995f * best) {
                best = ms;
                btws = sh[0];
                bm = sh[1];
            } else {
                e->tile_tws[g] = otws;
                e->tile_m[g] = om;
            }
        }
        e->tile_tws[g] = btws;
        e->tile_m[g] = bm;
        e->tiles_dirty = e->graph_dirty = true;
        const int g0 = e->grab[g];     // timed already
        int bg = g0;
        for (int gr : grabs) {
            if (rc) break;
            if (gr == g0) continue;
            e->grab[g] = gr;
            e->graph_dirty = true;
            if ((rc = time_schedule(e, a, b, &ms))) break;
            if (ms < 0.995f * best) {
                best = ms;
                bg = gr;
            } else {
                e->grab[g] = bg;
            }
        }
        e->grab[g] = bg;
        e->graph_dirty = true;
    }
    if (!rc) {
        const double bf = e->bps_factor;
        e->bps_factor = bf == 1.0 ? 0.5 : 1.0;
        e->graph_dirty = true;
        rc = time_schedule(e, a, b, &ms);
        if (!rc && ms >= 0.995f * best) e->bps_factor = bf;
        if (!rc && ms < 0.995f * best) best = ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc) return rc;
    e->graph_dirty = true;
    rc = prepare(e);
    if (best_ms_per_step) *best_ms_per_step = best / (2.0 * e->K);
    return rc;
}

namespace {

bool slot_group(const lbm_engine* e, int slot, int* g) {
    if (slot < 0 || slot >= e->max_slots || !e->slots[slot].used) return false;
    *g = e->slots[slot].group;
    return true;
}

}  // namespace

int lbm_engine_set_schedule(lbm_engine* e, int slot, int tile_width, int tile_cells, int grab,
                            double grid_fraction) {
    if (!e || e->pending) return LBM_EINVAL;
    if (tile_width != 0 && tile_width != 32 && tile_width != 64 && tile_width != 128) return LBM_EINVAL;
    if (tile_cells != 128 && tile_cells != 256 && tile_cells != 512) return LBM_EINVAL;
    if (grab < 1 || grab > 64 || !(grid_fraction > 0.0 && grid_fraction <= 1.0)) return LBM_EINVAL;
    int g0 = 0, g1 = kGroups;
    if (slot != -1) {
        if (!slot_group(e, slot, &g0)) return LBM_EINVAL;
        g1 = g0 + 1;
    }
    for (int g = g0; g < g1; ++g) {
        e->tile_tws[g] = tile_width == 0 ? 0 : (tile_width == 32 ? 5 : (tile_width == 64 ? 6 : 7));
        e->tile_m[g] = tile_cells / lbm::kBlock;
        e->grab[g] = grab;
    }
    e->bps_factor = grid_fraction;
    e->tiles_dirty = true;
    e->graph_dirty = true;
    return LBM_OK;
}

int lbm_engine_get_schedule(const lbm_engine* e, int slot, int* tile_width, int* tile_cells, int* grab,
                            double* grid_fraction) {
    int g = 0;
    if (!e || !slot_group(e, slot, &g)) return LBM_EINVAL;
    if (tile_width) *tile_width = e->tile_tws[g] ? 1 << e->tile_tws[g] : 0;
    if (tile_cells) *tile_cells = e->tile_m[g] * lbm::kBlock;
    if (grab) *grab = e->grab[g];
    if (grid_fraction) *grid_fraction = e->bps_factor;
    return LBM_OK;
}

int lbm_engine_info(lbm_engine* e, int slot, long* steps, int* status) {
    if (!e || slot < 0 || slot >= e->max_slots || !e->slots[slot].used) return LBM_EINVAL;
    if (steps) *steps = e->slots[slot].steps;
    if (status) {
        unsigned st = 0;
        cudaError_t err = cudaMemcpyAsync(&st, e->d_status + slot, sizeof(st), cudaMemcpyDeviceToHost,
                                          e->stream);
        if (err == cudaSuccess) err = cudaStreamSynchronize(e->stream);
        if (err != cudaSuccess) return cuda_rc(err);
        *status = st ? LBM_ENONFINITE : LBM_OK;
    }
    return LBM_OK;
}

int lbm_engine_moments(lbm_engine* e, int slot, double* rho, double* ux, double* uy) {
    if (!e || slot < 0 || slot >= e->max_slots || !e->slots[slot].used) return LBM_EINVAL;
    const EngSlot& h = e->slots[slot];
    const size_t n = size_t(e->slots[slot].spec.Nx) * e->slots[slot].spec.Ny * 8;
    cudaError_t err = cudaSuccess;
    if (rho) err = cudaMemcpyAsync(rho, h.rho, n, cudaMemcpyDeviceToHost, e->stream);
    if (ux && err == cudaSuccess) err = cudaMemcpyAsync(ux, h.ux, n, cudaMemcpyDeviceToHost, e->stream);
    if (uy && err == cudaSuccess) err = cudaMemcpyAsync(uy, h.uy, n, cudaMemcpyDeviceToHost, e->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(e->stream);
    return cuda_rc(err);
}

namespace {

struct EngineStateHeader {
    char magic[8];          // "LBMENG1\0"
    int V, Nx, Ny, precision, N, set_id;
    long steps;
    double tau, g;
};
static_assert(sizeof(EngineStateHeader) <= 64, "header fits its 64 bytes");

size_t engine_state_bytes(const EngSlot& sl) {
    const size_t n = size_t(sl.spec.Nx) * sl.spec.Ny;
    return 64 + size_t(sl.spec.V) * n * sl.spec.elem + 4 * n * 8;
}

}  // namespace

int lbm_engine_state_bytes(lbm_engine* e, int slot, size_t* bytes) {
    if (!e || !bytes || slot < 0 || slot >= e->max_slots || !e->slots[slot].used) return LBM_EINVAL;
    *bytes = engine_state_bytes(e->slots[slot]);
    return LBM_OK;
}

int lbm_engine_get_state(lbm_engine* e, int slot, void* host, size_t bytes) {
    if (!e || !host || slot < 0 || slot >= e->max_slots || !e->slots[slot].used) return LBM_EINVAL;
    const EngSlot& sl = e->slots[slot];
    if (bytes < engine_state_bytes(sl)) return LBM_EINVAL;
    const EngSlot& h = sl;
    const size_t n = size_t(sl.spec.Nx) * sl.spec.Ny, pb = size_t(sl.spec.V) * n * sl.spec.elem;
    EngineStateHeader hd{};
    std::memcpy(hd.magic, "LBMENG1", 8);
    hd.V = sl.spec.V;
    hd.Nx = sl.spec.Nx;
    hd.Ny = sl.spec.Ny;
    hd.precision = e->precision;
    hd.N = sl.spec.N;
    hd.set_id = sl.spec.set_id;
    hd.steps = sl.steps;
    hd.tau = h.tau;
    hd.g = h.g;
    char* out = static_cast<char*>(host);
    std::memset(out, 0, 64);
    std::memcpy(out, &hd, sizeof(hd));
    char* p = out + 64;
    cudaError_t err = cudaMemcpyAsync(p, h.f[h.phase], pb, cudaMemcpyDeviceToHost, e->stream);
    p += pb;
    const double* fields[4] = {h.rho, h.ux, h.uy, h.prev};
    for (int i = 0; i < 4 && err == cudaSuccess; ++i, p += n * 8)
        err = cudaMemcpyAsync(p, fields[i], n * 8, cudaMemcpyDeviceToHost, e->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(e->stream);
    return cuda_rc(err);
}

int lbm_engine_set_state(lbm_engine* e, int slot, const void* host, size_t bytes) {
    if (!e || !host || slot < 0 || slot >= e->max_slots || !e->slots[slot].used) return LBM_EINVAL;
    EngSlot& sl = e->slots[slot];
    if (bytes < engine_state_bytes(sl)) return LBM_EINVAL;
    EngineStateHeader hd{};
    std::memcpy(&hd, host, sizeof(hd));
    const EngSlot& h = sl;
    if (std::memcmp(hd.magic, "LBMENG1", 8) != 0 || hd.V != sl.spec.V || hd.Nx != sl.spec.Nx ||
        hd.Ny != sl.spec.Ny || hd.precision != e->precision || hd.N != sl.spec.N ||
        hd.set_id != sl.spec.set_id || hd.tau != h.tau || hd.g != h.g || hd.steps < 0)
        return LBM_EINVAL;
    const size_t n = size_t(sl.spec.Nx) * sl.spec.Ny, pb = size_t(sl.spec.V) * n * sl.spec.elem;
    const char* p = static_cast<const char*>(host) + 64;
    cudaError_t err = cudaMemcpyAsync(h.f[h.phase], p, pb, cudaMemcpyHostToDevice, e->stream);
    p += pb;
    double* fields[4] = {h.rho, h.ux, h.uy, h.prev};
    for (int i = 0; i < 4 && err == cudaSuccess; ++i, p += n * 8)
        err = cudaMemcpyAsync(fields[i], p, n * 8, cudaMemcpyHostToDevice, e->stream);
    if (err == cudaSuccess) err = cudaMemsetAsync(h.status, 0, sizeof(unsigned), e->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(e->stream);
    if (err == cudaSuccess) sl.steps = hd.steps;
    return cuda_rc(err);
}

int lbm_engine_free_bytes(lbm_engine* e, size_t* largest) {
    if (!e || !largest) return LBM_EINVAL;
    *largest = e->arena.largest();
    return LBM_OK;
}

}  // extern "C"
