// Merged launches for batched solves: the calling thread's launch recorder,
// the copy kernel that stands in for stream copies and fills while recording,
// and WaveRunner, which merges one wave of recorded launches of many
// independent problems into one launch per kernel and block size.
//
// Merge order: the records of each problem form a chain (problem order within
// a chain is stream order).  Repeatedly, among the next unmerged record of
// every problem, the kernel (with its block size) that the most problems wait
// on is taken; those problems' records become one merged launch (at most
// kMergeMax problems per launch), which depends on the launches that hold the
// same problems' previous records.  The result is a DAG of merged launches in
// which chains of different kernels (other degrees, other coarse-level
// structures) run concurrently, built as a CUDA graph.
#include "common.h"

#include <algorithm>
#include <cstdlib>
#include <mutex>
#include <unordered_map>

namespace hdg {

// launch family of this file for pdl_launch (Krylov and copy kernels)
constexpr unsigned kPdlFamily = 4;

bool pdl_enabled(unsigned family) {
    static const unsigned mask = [] {
        const char *e = std::getenv("HDG_PDL");
        return e ? unsigned(std::strtoul(e, nullptr, 0)) : 6u;
    }();
    return (mask & family) != 0;
}

Recorder *&batch_recorder() {
    static thread_local Recorder *r = nullptr;
    return r;
}

namespace {

inline unsigned blocks(size_t n, int bs) { return unsigned((n + bs - 1) / bs); }

// dst[0, n) = src[0, n) (src null: zeros), in 8-byte words when both
// addresses and n allow it
__device__ __forceinline__ void copy_kernel_impl(int bid_, int nb_, unsigned char *dst, const unsigned char *src,
                                                 size_t n) {
    const size_t t = size_t(bid_) * blockDim.x + threadIdx.x, stride = size_t(nb_) * blockDim.x;
    if (((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src) | n) & 7) == 0) {
        uint64_t *d = reinterpret_cast<uint64_t *>(dst);
        const uint64_t *s = reinterpret_cast<const uint64_t *>(src);
        for (size_t i = t; i < n / 8; i += stride) d[i] = s ? s[i] : 0ull;
    } else {
        for (size_t i = t; i < n; i += stride) dst[i] = src ? src[i] : static_cast<unsigned char>(0);
    }
}
__global__ void copy_kernel(unsigned char *dst, const unsigned char *src, size_t n) {
    pdl_wait();
    copy_kernel_impl(blockIdx.x, gridDim.x, dst, src, n);
}
struct copy_kernel_args {
    int nb_;
    unsigned char *dst;
    const unsigned char *src;
    size_t n;
};
__global__ void copy_kernel_multi(const __grid_constant__ MultiP<copy_kernel_args> M) {
    pdl_wait();
    int b_;
    const copy_kernel_args &q_ = M.a[merge_find(M.start, M.n, b_)];
    copy_kernel_impl(b_, q_.nb_, q_.dst, q_.src, q_.n);
}
void copy_kernel_go(unsigned grid_, unsigned block_, size_t smem_, cudaStream_t s_, unsigned char *dst,
                    const unsigned char *src, size_t n) {
    if (Recorder *r_ = batch_recorder()) {
        copy_kernel_args q_;
        std::memset(static_cast<void *>(&q_), 0, sizeof(q_));
        q_.nb_ = int(grid_);
        q_.dst = dst;
        q_.src = src;
        q_.n = n;
        batch_record(r_, reinterpret_cast<const void *>(&copy_kernel_multi), q_, grid_, block_, smem_, kPdlFamily);
        return;
    }
    pdl_launch(kPdlFamily, &copy_kernel, grid_, block_, smem_, s_, dst, src, n);
}


// 64-bit hash of a byte string, eight bytes at a time
uint64_t hash_bytes(const unsigned char *p, size_t n) {
    uint64_t h = 0x9e3779b97f4a7c15ull ^ n;
    size_t i = 0;
    for (; i + 8 <= n; i += 8) {
        uint64_t w;
        std::memcpy(&w, p + i, 8);
        w *= 0xff51afd7ed558ccdull;
        w ^= w >> 32;
        h = (h ^ w) * 0xc4ceb9fe1a85ec53ull;
        h ^= h >> 29;
    }
    for (; i < n; ++i) h = (h ^ p[i]) * 0x100000001b3ull;
    return h ^ (h >> 31);
}

// dynamic shared memory limits raised so far, per merged kernel (the
// attribute is process-wide and only ever raised here)
std::mutex g_attr_mu;
std::unordered_map<const void *, size_t> g_attr;

cudaError_t ensure_smem_limit(const void *func, size_t smem) {
    if (smem <= 48 * 1024) return cudaSuccess;
    std::lock_guard<std::mutex> lk(g_attr_mu);
    size_t &cur = g_attr[func];
    if (cur >= smem) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e == cudaSuccess) cur = smem;
    return e;
}

}  // namespace

cudaError_t launch_copy(void *dst, const void *src, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const unsigned nb = std::min<unsigned>(blocks((n + 7) / 8, 256), 1216);
    copy_kernel_go(nb, 256, 0, s, static_cast<unsigned char *>(dst), static_cast<const unsigned char *>(src), n);
    return cudaGetLastError();
}

void WaveRunner::clear() {
    for (auto &b : buckets_) {
        for (auto &e : b)
            if (e.exec) cudaGraphExecDestroy(e.exec);
        b.clear();
    }
    key_bytes_ = 0;
}

cudaError_t WaveRunner::build(Recorder *const *recs, int n, Entry &out) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return e;
    std::vector<size_t> head(size_t(n), 0);
    std::vector<cudaGraphNode_t> last(size_t(n), nullptr);
    std::vector<unsigned char> param;
    std::vector<int> start, group;
    std::vector<const unsigned char *> argp;
    std::vector<cudaGraphNode_t> deps;
    struct Sig {
        const void *func;
        unsigned block;
        bool operator==(const Sig &o) const { return func == o.func && block == o.block; }
    };
    for (;;) {
        // the signature most problems wait on next (ties: the earliest problem's)
        std::vector<std::pair<Sig, int>> count;
        for (int i = 0; i < n; ++i) {
            const Recorder &r = *recs[i];
            while (head[i] < r.recs.size() && r.recs[head[i]].grid == 0) ++head[i];
            if (head[i] >= r.recs.size()) continue;
            const Sig sg{r.recs[head[i]].func, r.recs[head[i]].block};
            auto it = std::find_if(count.begin(), count.end(), [&](const std::pair<Sig, int> &c) { return c.first == sg; });
            if (it == count.end()) count.push_back({sg, 1});
            else ++it->second;
        }
        if (count.empty()) break;
        const Sig pick = std::max_element(count.begin(), count.end(), [](const std::pair<Sig, int> &a,
                                                                          const std::pair<Sig, int> &b) {
                             return a.second < b.second;
                         })->first;
        group.clear();
        for (int i = 0; i < n; ++i) {
            const Recorder &r = *recs[i];
            if (head[i] < r.recs.size() && Sig{r.recs[head[i]].func, r.recs[head[i]].block} == pick) group.push_back(i);
        }
        for (size_t g0 = 0; g0 < group.size(); g0 += kMergeMax) {
            const int m = int(std::min<size_t>(kMergeMax, group.size() - g0));
            start.assign(size_t(m) + 1, 0);
            argp.assign(size_t(m), nullptr);
            deps.clear();
            size_t smem = 0;
            const MergeRec *r0 = nullptr;
            for (int q = 0; q < m; ++q) {
                const int i = group[g0 + size_t(q)];
                const MergeRec &rc = recs[i]->recs[head[i]];
                r0 = &rc;
                if (uint64_t(start[size_t(q)]) + rc.grid > uint64_t(0x7fffffff)) {
                    cudaGraphDestroy(g);
                    return cudaErrorInvalidConfiguration;
                }
                start[size_t(q) + 1] = start[size_t(q)] + int(rc.grid);
                argp[size_t(q)] = recs[i]->arena.data() + rc.off;
                smem = std::max(smem, rc.smem);
                if (last[size_t(i)] && std::find(deps.begin(), deps.end(), last[size_t(i)]) == deps.end())
                    deps.push_back(last[size_t(i)]);
            }
            param.assign(r0->param_bytes, 0);
            r0->pack(param.data(), m, start.data(), argp.data());
            if ((e = ensure_smem_limit(r0->func, smem)) != cudaSuccess) {
                cudaGraphDestroy(g);
                return e;
            }
            void *kargs[1] = {param.data()};
            cudaKernelNodeParams kp{};
            kp.func = const_cast<void *>(r0->func);
            kp.gridDim = dim3(unsigned(start[size_t(m)]));
            kp.blockDim = dim3(r0->block);
            kp.sharedMemBytes = unsigned(smem);
            kp.kernelParams = kargs;
            kp.extra = nullptr;
            cudaGraphNode_t node = nullptr;
            if ((e = cudaGraphAddKernelNode(&node, g, nullptr, 0, &kp)) != cudaSuccess) {
                cudaGraphDestroy(g);
                return e;
            }
            // edges from the launches that hold the same problems' previous
            // records: programmatic for the families launched that way in
            // single solves (the merged kernels wait for their predecessors in
            // griddepcontrol.wait), full dependencies otherwise
            cudaGraphEdgeData ed{};
            if (pdl_enabled(r0->family)) {
                ed.from_port = cudaGraphKernelNodePortProgrammatic;
                ed.type = cudaGraphDependencyTypeProgrammatic;
            }
            for (cudaGraphNode_t d : deps)
                if ((e = cudaGraphAddDependencies(g, &d, &node, &ed, 1)) != cudaSuccess) {
                    cudaGraphDestroy(g);
                    return e;
                }
            out.nodes += 1;
            out.records += m;
            for (int q = 0; q < m; ++q) {
                const int i = group[g0 + size_t(q)];
                last[size_t(i)] = node;
                ++head[size_t(i)];
            }
        }
    }
    e = cudaGraphInstantiate(&out.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) out.exec = nullptr;
    return e;
}

cudaError_t WaveRunner::run(Recorder *const *recs, int n, cudaStream_t s) {
    // the key: per problem, its index, record count and every record in full
    key_.clear();
    auto put = [this](const void *p, size_t b) {
        const unsigned char *c = static_cast<const unsigned char *>(p);
        key_.insert(key_.end(), c, c + b);
    };
    bool any = false;
    for (int i = 0; i < n; ++i) {
        const Recorder &r = *recs[i];
        if (r.recs.empty()) continue;
        any = true;
        const int32_t hdr[2] = {i, int32_t(r.recs.size())};
        put(hdr, sizeof(hdr));
        for (const MergeRec &m : r.recs) {
            put(&m.func, sizeof(m.func));
            const uint64_t shape[3] = {m.grid, m.block, m.smem};
            put(shape, sizeof(shape));
            put(r.arena.data() + m.off, m.args_bytes);
        }
    }
    if (!any) return cudaSuccess;
    const uint64_t hv = hash_bytes(key_.data(), key_.size());
    std::vector<Entry> &bucket = buckets_[hv % buckets_.size()];
    stats.waves += 1;
    for (Entry &en : bucket) {
        if (en.key.size() == key_.size() && std::memcmp(en.key.data(), key_.data(), key_.size()) == 0) {
            stats.hits += 1;
            stats.nodes += en.nodes;
            stats.records += en.records;
            return cudaGraphLaunch(en.exec, s);
        }
    }
    // a new wave: keep at most 256 MB of keys, then start over
    if (key_bytes_ + key_.size() > (size_t(256) << 20)) clear();
    Entry en;
    cudaError_t e = build(recs, n, en);
    if (e != cudaSuccess) return e;
    stats.misses += 1;
    stats.nodes += en.nodes;
    stats.records += en.records;
    en.key = key_;
    key_bytes_ += en.key.size();
    std::vector<Entry> &b2 = buckets_[hv % buckets_.size()];
    b2.push_back(std::move(en));
    return cudaGraphLaunch(b2.back().exec, s);
}

}  // namespace hdg
