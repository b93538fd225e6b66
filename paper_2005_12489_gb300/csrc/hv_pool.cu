// Result pool: HiVision's IMMF Result Pool (Sec. 4.2), a key-value store of
// rendered tiles with expiry, which lets Parse Tasks (Sec. 4.1) drop a
// request whose tile is already rendered.  Here it is a host-memory LRU cache
// keyed by (layer, z, x, y, r16, mode, style) under a byte capacity, with an
// optional time to live.  Host code only: the serving loop consults it at
// submission and fills it as batches complete; callers of hv_render_tiles
// may use it the same way.
#include <string.h>

#include <chrono>
#include <list>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "hv_internal.h"

namespace hv {

namespace {

struct PoolKey {
    uint32_t layer, x, y;
    uint16_t r16;
    uint8_t z, mode;
    uint8_t style[8];   // zero unless the mode is RGBA (colours change only RGBA)
    bool operator==(const PoolKey& o) const { return memcmp(this, &o, sizeof(PoolKey)) == 0; }
};
static_assert(sizeof(PoolKey) == 24, "packed key");

struct PoolKeyHash {
    size_t operator()(const PoolKey& k) const {
        uint64_t w[3];
        memcpy(w, &k, sizeof(w));
        uint64_t h = w[0] * 0x9E3779B97F4A7C15ull;
        h ^= (w[1] + 0x632BE59BD9B4E019ull + (h << 6) + (h >> 2)) * 0xBF58476D1CE4E5B9ull;
        h ^= (w[2] + 0x94D049BB133111EBull + (h << 6) + (h >> 2)) * 0x94D049BB133111EBull;
        return (size_t)(h ^ (h >> 31));
    }
};

PoolKey make_key(const hv_tile_req& r, const hv_style* style) {
    PoolKey k;
    memset(&k, 0, sizeof(k));
    k.layer = r.layer;
    k.x = r.x;
    k.y = r.y;
    k.r16 = r.r16;
    k.z = r.z;
    k.mode = r.mode;
    if (r.mode == HV_MODE_RGBA && style) memcpy(k.style, style, 8);
    return k;
}

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct ResultPool {
    struct Entry {
        std::vector<uint8_t> data;
        double t_insert;
        std::list<PoolKey>::iterator lru;
    };
    uint64_t capacity = 0;
    double ttl_ms = 0;   // 0: no expiry
    std::mutex mu;
    std::unordered_map<PoolKey, Entry, PoolKeyHash> map;
    std::list<PoolKey> lru;   // front: most recently used
    uint64_t bytes = 0;
    hv_pool_stats st{};

    bool expired(const Entry& e, double t) const { return ttl_ms > 0 && t - e.t_insert > ttl_ms; }

    void drop(std::unordered_map<PoolKey, Entry, PoolKeyHash>::iterator it) {
        bytes -= it->second.data.size();
        lru.erase(it->second.lru);
        map.erase(it);
    }

    // Evict from the least recently used end until `need` more bytes fit.
    void make_room(uint64_t need, double t) {
        while (bytes + need > capacity && !lru.empty()) {
            auto it = map.find(lru.back());
            if (expired(it->second, t))
                st.expirations++;
            else
                st.evictions++;
            drop(it);
        }
    }
};

// The serving loop's use of a pool (hv_server.cu).
bool pool_lookup(ResultPool* P, const hv_tile_req& r, const hv_style* style, std::vector<uint8_t>* out) {
    std::lock_guard<std::mutex> g(P->mu);
    auto it = P->map.find(make_key(r, style));
    const double t = now_ms();
    if (it == P->map.end() || P->expired(it->second, t)) {
        if (it != P->map.end()) {
            P->st.expirations++;
            P->drop(it);
        }
        P->st.misses++;
        return false;
    }
    *out = it->second.data;
    P->lru.splice(P->lru.begin(), P->lru, it->second.lru);
    P->st.hits++;
    return true;
}

int pool_insert(ResultPool* P, const hv_tile_req& r, const hv_style* style, const void* data, uint64_t n) {
    std::lock_guard<std::mutex> g(P->mu);
    if (n > P->capacity) {
        P->st.rejected++;
        set_error("result pool: a %llu-byte tile exceeds the capacity of %llu bytes", (unsigned long long)n,
                  (unsigned long long)P->capacity);
        return HV_ENOMEM;
    }
    const PoolKey k = make_key(r, style);
    const double t = now_ms();
    auto it = P->map.find(k);
    if (it != P->map.end()) P->drop(it);
    P->make_room(n, t);
    ResultPool::Entry e;
    e.data.assign((const uint8_t*)data, (const uint8_t*)data + n);
    e.t_insert = t;
    P->lru.push_front(k);
    e.lru = P->lru.begin();
    P->map.emplace(k, std::move(e));
    P->bytes += n;
    P->st.inserts++;
    return HV_OK;
}

}  // namespace hv

using namespace hv;

extern "C" {

int hv_result_pool_create(uint64_t capacity_bytes, uint32_t ttl_ms, hv_result_pool** out) {
    if (!out || capacity_bytes == 0) { set_error("hv_result_pool_create: NULL out or zero capacity"); return HV_EINVAL; }
    ResultPool* P = new ResultPool();
    P->capacity = capacity_bytes;
    P->ttl_ms = ttl_ms;
    *out = (hv_result_pool*)P;
    return HV_OK;
}

int hv_result_pool_destroy(hv_result_pool* pool) {
    if (!pool) return HV_EINVAL;
    delete (ResultPool*)pool;
    return HV_OK;
}

int hv_result_pool_put(hv_result_pool* pool, const hv_tile_req* req, const hv_style* style, const void* data,
                       uint64_t bytes) {
    if (!pool || !req || (!data && bytes)) { set_error("hv_result_pool_put: NULL argument"); return HV_EINVAL; }
    return pool_insert((ResultPool*)pool, *req, style, data, bytes);
}

int hv_result_pool_get(hv_result_pool* pool, const hv_tile_req* req, const hv_style* style, void* out,
                       uint64_t out_bytes, uint32_t* hit) {
    if (!pool || !req || !hit) { set_error("hv_result_pool_get: NULL argument"); return HV_EINVAL; }
    std::vector<uint8_t> v;
    *hit = 0;
    if (!pool_lookup((ResultPool*)pool, *req, style, &v)) return HV_OK;
    if (!out || out_bytes < v.size()) {
        set_error("hv_result_pool_get: out_bytes %llu < %llu", (unsigned long long)out_bytes,
                  (unsigned long long)v.size());
        return HV_EINVAL;
    }
    memcpy(out, v.data(), v.size());
    *hit = 1;
    return HV_OK;
}

int hv_result_pool_stats(hv_result_pool* pool, hv_pool_stats* out) {
    if (!pool || !out) { set_error("hv_result_pool_stats: NULL argument"); return HV_EINVAL; }
    ResultPool* P = (ResultPool*)pool;
    std::lock_guard<std::mutex> g(P->mu);
    *out = P->st;
    out->entries = P->map.size();
    out->bytes = P->bytes;
    out->capacity = P->capacity;
    return HV_OK;
}

int hv_result_pool_clear(hv_result_pool* pool) {
    if (!pool) return HV_EINVAL;
    ResultPool* P = (ResultPool*)pool;
    std::lock_guard<std::mutex> g(P->mu);
    P->map.clear();
    P->lru.clear();
    P->bytes = 0;
    return HV_OK;
}

}  // extern "C"
