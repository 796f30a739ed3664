// hj_debug.cu -- the library's device allocations, and what debug builds add
// around them as a stand-in for a memory checker:
//   * guard bands: every device allocation of the library (handle workspaces)
//     gets kGuard bytes of a fixed pattern on each side;
//   * the index-check word: kernels of debug builds check their staging,
//     exchange and write-back indices (HJ_IN) and record the first failure
//     here instead of trapping;
//   * hj_debug_check reports both, hj_debug_selftest shows that each is
//     caught, without touching memory out of bounds.
// Release builds allocate with plain cudaMalloc / cudaFree, compile the index
// checks away, and hj_debug_check reports that no checks are compiled in.
#include <map>
#include <mutex>

#include "hj_runtime.cuh"

namespace hj {

namespace {

#ifdef HJ_DEBUG
constexpr size_t kGuard = 256;   // bytes on each side (keeps 256-byte alignment)
constexpr unsigned char kPattern = 0xA5;

struct Alloc {
    unsigned char *base;   // start of the leading guard
    size_t bytes;          // bytes handed out
};
std::mutex g_mu;
std::map<void *, Alloc> g_allocs;
DbgWord *g_word = nullptr;

// The first byte of either guard band of a that no longer holds the pattern:
// its offset from the start of the bytes handed out (negative: before them).
bool guard_broken(void *user, const Alloc &a, long long *offset) {
    unsigned char buf[2][kGuard];
    if (cudaMemcpy(buf[0], a.base, kGuard, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(buf[1], (unsigned char *)user + a.bytes, kGuard, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        *offset = 0;
        return true;
    }
    for (size_t i = 0; i < kGuard; ++i) {
        if (buf[0][i] != kPattern) {
            *offset = (long long)i - (long long)kGuard;
            return true;
        }
        if (buf[1][i] != kPattern) {
            *offset = (long long)(a.bytes + i);
            return true;
        }
    }
    return false;
}

__global__ void debug_selftest_kernel(DbgWord *w) {
    // one index inside [0, 4) and one outside it: the check records the
    // second, and neither addresses any memory
    (void)HJ_IN(w, 3, 4, 998);
    (void)HJ_IN(w, 5, 4, 999);
}
#endif

}  // namespace

cudaError_t dmalloc(void **p, size_t bytes) {
#ifdef HJ_DEBUG
    unsigned char *base = nullptr;
    cudaError_t e = cudaMalloc((void **)&base, bytes + 2 * kGuard);
    if (e != cudaSuccess) {
        *p = nullptr;
        return e;
    }
    e = cudaMemset(base, kPattern, kGuard);
    if (e == cudaSuccess) e = cudaMemset(base + kGuard + bytes, kPattern, kGuard);
    if (e != cudaSuccess) {
        cudaFree(base);
        *p = nullptr;
        return e;
    }
    *p = base + kGuard;
    std::lock_guard<std::mutex> lk(g_mu);
    g_allocs[*p] = Alloc{base, bytes};
    return cudaSuccess;
#else
    return cudaMalloc(p, bytes);
#endif
}

cudaError_t dfree(void *p) {
    if (!p) return cudaSuccess;
#ifdef HJ_DEBUG
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_allocs.find(p);
    if (it == g_allocs.end()) return cudaFree(p);
    unsigned char *base = it->second.base;
    g_allocs.erase(it);
    return cudaFree(base);
#else
    return cudaFree(p);
#endif
}

DbgWord *debug_word() {
#ifdef HJ_DEBUG
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_word) {
        if (cudaMalloc((void **)&g_word, sizeof(DbgWord)) != cudaSuccess ||
            cudaMemset(g_word, 0, sizeof(DbgWord)) != cudaSuccess) {
            cudaGetLastError();
            g_word = nullptr;
        }
    }
    return g_word;
#else
    return nullptr;
#endif
}

}  // namespace hj

using namespace hj;

extern "C" int hj_debug_check(long long *site, long long *index) {
    long long s = 0, i = 0;
#ifdef HJ_DEBUG
    CKR(cudaDeviceSynchronize());
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (g_word) {
            DbgWord w;
            CKR(cudaMemcpy(&w, g_word, sizeof(w), cudaMemcpyDeviceToHost));
            if (w.site) {
                s = (long long)w.site;
                i = w.index;
                CKR(cudaMemset(g_word, 0, sizeof(DbgWord)));
            }
        }
        if (!s) {
            for (auto &kv : g_allocs) {
                long long off = 0;
                if (guard_broken(kv.first, kv.second, &off)) {
                    s = -2;
                    i = off;
                    // restore the pattern, so that one breach is reported once
                    cudaMemset(kv.second.base, kPattern, kGuard);
                    cudaMemset((unsigned char *)kv.first + kv.second.bytes, kPattern, kGuard);
                    break;
                }
            }
        }
    }
#else
    s = -1;   // no checks compiled in
#endif
    if (site) *site = s;
    if (index) *index = i;
    if (s > 0) return seterr(HJ_ERR_BOUNDS, "debug check: index %lld out of range at kernel site %lld", i, s);
    if (s == -2) return seterr(HJ_ERR_BOUNDS, "debug check: guard band overwritten at byte offset %lld", i);
    return HJ_OK;
}

extern "C" int hj_debug_selftest(void) {
#ifdef HJ_DEBUG
    long long s = 0, i = 0;
    // a clean start
    hj_debug_check(&s, &i);
    // 1. the index check of a kernel
    DbgWord *w = debug_word();
    if (!w) return seterr(HJ_ERR_CUDA, "debug word not allocated");
    debug_selftest_kernel<<<1, 1>>>(w);
    CKR(cudaGetLastError());
    const int st1 = hj_debug_check(&s, &i);
    const bool index_caught = st1 == HJ_ERR_BOUNDS && s == 999 && i == 5;
    // 2. a guard band: the byte 17 past the end of a 1000-byte allocation,
    //    written by the host (inside the allocation with its guards)
    void *p = nullptr;
    CKR(dmalloc(&p, 1000));
    const int st0 = hj_debug_check(&s, &i);
    CKR(cudaMemset((unsigned char *)p + 1000 + 17, 0, 1));
    const int st2 = hj_debug_check(&s, &i);
    const bool guard_caught = st0 == HJ_OK && st2 == HJ_ERR_BOUNDS && s == -2 && i == 1017;
    CKR(dfree(p));
    if (!index_caught || !guard_caught)
        return seterr(HJ_ERR_BOUNDS, "debug self-test: index check %s, guard band %s",
                      index_caught ? "caught" : "missed", guard_caught ? "caught" : "missed");
    return HJ_OK;
#else
    return seterr(HJ_ERR_UNSUPPORTED, "hj_debug_selftest: this library was built without HJ_DEBUG");
#endif
}
