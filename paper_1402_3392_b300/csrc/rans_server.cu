// rans_server.cu -- continuous-batching request loop over the batched coder.
//
// The server owns one device arena (the caller's HBM budget) and a few
// "slots", each a CUDA stream with page-locked staging buffers.  It replays a
// trace of requests in real time:
//   - a request becomes pending at its arrival time;
//   - pending requests are admitted in arrival order while their device input
//     and output fit in the arena (first fit, 256-byte granules); a request
//     larger than the whole arena fails with RANS_ERR_OOM;
//   - admitted requests go into the next idle slot as one batch: host-to-device
//     copies of the inputs, one rans_encode_batch and/or one rans_decode_batch
//     launch (the models stay resident in d_freqs), then device-to-host copies
//     of the statuses, sizes and outputs (an encoded message's size is known
//     only after its kernel, so its copy is issued once the slot reports it);
//   - while one slot's batch runs, newer arrivals are admitted into the other
//     slots as memory frees up, so copies and kernels of different batches
//     overlap on the device;
//   - a request is done when its output is in host memory; its device memory
//     is released then;
//   - a request flagged RANS_REQ_DEVICE_MEMORY carries device input and output
//     buffers: the coders read and write them in place, nothing is copied and
//     only the batch's scratch and descriptors take arena memory; it is done
//     when its kernels are.
// All device work goes through the library's batched entry points; this file
// is host code only.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "host_util.h"

namespace rans {
namespace {

constexpr uint64_t kGranule = 256;

uint64_t up(uint64_t v) { return (std::max<uint64_t>(v, 1) + kGranule - 1) / kGranule * kGranule; }

// First-fit allocator over [0, bytes) with coalescing of free ranges.
class Arena {
  public:
    explicit Arena(uint64_t bytes) : bytes_(bytes) { free_[0] = bytes; }
    bool alloc(uint64_t n, uint64_t *off) {
        n = up(n);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            const uint64_t o = it->first, rest = it->second - n;
            free_.erase(it);
            if (rest) free_[o + n] = rest;
            *off = o;
            used_ += n;
            return true;
        }
        return false;
    }
    void release(uint64_t off, uint64_t n) {
        n = up(n);
        used_ -= n;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + n == next->first) {
            n += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += n;
                return;
            }
        }
        free_[off] = n;
    }
    uint64_t bytes() const { return bytes_; }

  private:
    uint64_t bytes_, used_ = 0;
    std::map<uint64_t, uint64_t> free_;
};

struct Req {
    uint32_t id;
    uint64_t in_off, in_len, out_off, out_len;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    int phase = 0;  // 0 idle, 1 kernels in flight, 2 output copies in flight
    uint32_t batch = 0;
    std::vector<Req> enc, dec;
    std::vector<std::pair<uint64_t, uint64_t>> batch_allocs;  // (offset, bytes)
    // page-locked staging
    rans_encode_stream *h_enc = nullptr;
    rans_stream *h_dec = nullptr;
    uint64_t *h_sizes = nullptr;
    uint32_t *h_status = nullptr;
};

struct Server {
    const uint16_t *d_freqs;
    uint32_t n_tables;
    uint8_t *d_arena;
    Arena arena;
    uint32_t max_batch;
    std::vector<Slot> slots;
    Server(uint64_t bytes) : arena(bytes) {}
};

double seconds_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

uint32_t request_kind(const rans_request &r) { return r.kind & ~RANS_REQ_DEVICE_MEMORY; }
bool on_device(const rans_request &r) { return (r.kind & RANS_REQ_DEVICE_MEMORY) != 0; }

uint64_t request_output_bytes(const rans_request &r) {
    if (request_kind(r) == RANS_REQ_ENCODE) {
        rans_params p{r.n_lanes, r.chunk_symbols};
        return rans_max_encoded_size(r.n_symbols, &p);
    }
    return r.n_symbols;
}

}  // namespace
}  // namespace rans

using namespace rans;

extern "C" int rans_server_create(const uint16_t *d_freqs, uint32_t n_tables, void *d_arena,
                                  uint64_t arena_bytes, uint32_t max_batch, uint32_t n_slots,
                                  rans_server **out) {
    if (!out || !d_freqs || n_tables == 0 || !d_arena || !aligned16(d_arena) ||
        arena_bytes < 4 * kGranule || max_batch == 0 || n_slots == 0 || n_slots > 16)
        return RANS_ERR_INVALID_ARG;
    *out = nullptr;
    Server *s = new Server(arena_bytes / kGranule * kGranule);
    s->d_freqs = d_freqs;
    s->n_tables = n_tables;
    s->d_arena = static_cast<uint8_t *>(d_arena);
    s->max_batch = max_batch;
    s->slots.resize(n_slots);
    for (Slot &sl : s->slots) {
        bool ok = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) == cudaSuccess &&
                  cudaMallocHost(&sl.h_enc, sizeof(rans_encode_stream) * max_batch) == cudaSuccess &&
                  cudaMallocHost(&sl.h_dec, sizeof(rans_stream) * max_batch) == cudaSuccess &&
                  cudaMallocHost(&sl.h_sizes, sizeof(uint64_t) * max_batch) == cudaSuccess &&
                  cudaMallocHost(&sl.h_status, sizeof(uint32_t) * 2 * max_batch) == cudaSuccess;
        if (!ok) {
            rans_server_destroy(reinterpret_cast<rans_server *>(s));
            return RANS_ERR_CUDA;
        }
    }
    *out = reinterpret_cast<rans_server *>(s);
    return RANS_OK;
}

extern "C" void rans_server_destroy(rans_server *srv) {
    Server *s = reinterpret_cast<Server *>(srv);
    if (!s) return;
    for (Slot &sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.h_enc) cudaFreeHost(sl.h_enc);
        if (sl.h_dec) cudaFreeHost(sl.h_dec);
        if (sl.h_sizes) cudaFreeHost(sl.h_sizes);
        if (sl.h_status) cudaFreeHost(sl.h_status);
    }
    delete s;
}

extern "C" int rans_server_run(rans_server *srv, const rans_request *reqs, uint32_t n,
                               rans_result *results) {
    Server *s = reinterpret_cast<Server *>(srv);
    if (!s || (n && (!reqs || !results))) return RANS_ERR_INVALID_ARG;
    for (uint32_t i = 0; i < n; ++i) {
        const rans_request &r = reqs[i];
        rans_params p{r.n_lanes, r.chunk_symbols};
        std::memset(&results[i], 0, sizeof(rans_result));
        const uint32_t kind = request_kind(r);
        if ((kind != RANS_REQ_ENCODE && kind != RANS_REQ_DECODE) || !params_ok(&p) ||
            r.table >= s->n_tables || (r.input_size && !r.input) || !r.output ||
            r.output_cap < request_output_bytes(r) ||
            (kind == RANS_REQ_ENCODE && r.input_size != r.n_symbols) ||
            (kind == RANS_REQ_DECODE && (r.input_size & 15u)) ||
            // device payloads are read and written in place: a message and an
            // encode output must be 16-byte aligned, as for the coders
            (on_device(r) && kind == RANS_REQ_DECODE && !aligned16(r.input)) ||
            (on_device(r) && kind == RANS_REQ_ENCODE && !aligned16(r.output)) ||
            (i && r.arrival_s < reqs[i - 1].arrival_s))
            return RANS_ERR_INVALID_ARG;
    }
    const auto t0 = std::chrono::steady_clock::now();
    std::deque<uint32_t> pending;
    uint32_t next = 0, done = 0, batches = 0;
    int rc = RANS_OK;

    // A request's input and output regions in the arena (none for device
    // payloads, which the coders read and write in place).
    auto release_payload = [&](const Req &q) {
        if (on_device(reqs[q.id])) return;
        s->arena.release(q.in_off, q.in_len);
        s->arena.release(q.out_off, q.out_len);
    };
    auto place_payload = [&](Req &q) {
        if (on_device(reqs[q.id])) return true;
        if (!s->arena.alloc(q.in_len, &q.in_off)) return false;
        if (!s->arena.alloc(q.out_len, &q.out_off)) {
            s->arena.release(q.in_off, q.in_len);
            return false;
        }
        return true;
    };
    auto input_of = [&](const Req &q) -> const uint8_t * {
        return on_device(reqs[q.id]) ? reqs[q.id].input : s->d_arena + q.in_off;
    };
    auto output_of = [&](const Req &q) -> uint8_t * {
        return on_device(reqs[q.id]) ? reqs[q.id].output : s->d_arena + q.out_off;
    };

    auto finish = [&](Slot &sl) {
        const double t = seconds_since(t0);
        for (size_t k = 0; k < sl.enc.size(); ++k) {
            const Req &q = sl.enc[k];
            results[q.id].status = sl.h_status[k];
            results[q.id].output_size = sl.h_status[k] == RANS_OK ? sl.h_sizes[k] : 0;
            results[q.id].done_s = t;
            release_payload(q);
        }
        for (size_t k = 0; k < sl.dec.size(); ++k) {
            const Req &q = sl.dec[k];
            const uint32_t st = sl.h_status[s->max_batch + k];
            results[q.id].status = st;
            results[q.id].output_size = st == RANS_OK ? reqs[q.id].n_symbols : 0;
            results[q.id].done_s = t;
            release_payload(q);
        }
        for (auto &a : sl.batch_allocs) s->arena.release(a.first, a.second);
        done += uint32_t(sl.enc.size() + sl.dec.size());
        sl.enc.clear();
        sl.dec.clear();
        sl.batch_allocs.clear();
        sl.phase = 0;
    };

    while (done < n && rc == RANS_OK) {
        bool progressed = false;
        const double now = seconds_since(t0);
        while (next < n && reqs[next].arrival_s <= now) pending.push_back(next++);

        // completions
        for (Slot &sl : s->slots) {
            if (sl.phase == 0) continue;
            const cudaError_t q = cudaEventQuery(sl.ev);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) {
                rc = RANS_ERR_CUDA;
                break;
            }
            progressed = true;
            const bool copy_out = std::any_of(sl.enc.begin(), sl.enc.end(), [&](const Req &q) {
                return !on_device(reqs[q.id]);
            });
            if (sl.phase == 1 && copy_out) {
                // encoded sizes are known now: copy the messages out
                for (size_t k = 0; k < sl.enc.size(); ++k) {
                    if (sl.h_status[k] != RANS_OK) continue;
                    const Req &qq = sl.enc[k];
                    if (on_device(reqs[qq.id])) continue;
                    if (cudaMemcpyAsync(reqs[qq.id].output, s->d_arena + qq.out_off, sl.h_sizes[k],
                                        cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess)
                        rc = RANS_ERR_CUDA;
                }
                if (cudaEventRecord(sl.ev, sl.stream) != cudaSuccess) rc = RANS_ERR_CUDA;
                sl.phase = 2;
            } else {
                finish(sl);
            }
        }

        // admission into idle slots
        for (Slot &sl : s->slots) {
            if (rc != RANS_OK || pending.empty()) break;
            if (sl.phase != 0) continue;
            std::vector<Req> enc, dec;
            while (!pending.empty() && enc.size() + dec.size() < s->max_batch) {
                const uint32_t id = pending.front();
                const rans_request &r = reqs[id];
                Req q{id, 0, r.input_size, 0, request_output_bytes(r)};
                if (!on_device(r) && up(q.in_len) + up(q.out_len) > s->arena.bytes()) {
                    results[id].status = RANS_ERR_OOM;  // can never fit
                    results[id].admit_s = results[id].done_s = seconds_since(t0);
                    pending.pop_front();
                    ++done;
                    progressed = true;
                    continue;
                }
                if (!place_payload(q)) break;
                pending.pop_front();
                (request_kind(r) == RANS_REQ_ENCODE ? enc : dec).push_back(q);
            }
            if (enc.empty() && dec.empty()) break;
            // Batch-level regions: encode scratch, decode scratch, descriptors,
            // results -- all or nothing.  If they do not fit, retry with the
            // head request alone; if even that does not fit while nothing is
            // in flight to free memory, the head request can never run.
            uint64_t need[4], offs[4];
            auto plan_batch = [&]() {
                for (size_t k = 0; k < enc.size(); ++k) {
                    const rans_request &r = reqs[enc[k].id];
                    rans_encode_stream &d = sl.h_enc[k];
                    d.symbols = input_of(enc[k]);
                    d.n_symbols = r.n_symbols;
                    d.out = output_of(enc[k]);
                    d.out_cap = enc[k].out_len;
                    d.scratch_offset = 0;
                    d.table = r.table;
                    d.n_lanes = r.n_lanes;
                    d.chunk_symbols = r.chunk_symbols;
                    d.reserved = 0;
                }
                need[0] = enc.empty() ? 0 : rans_encode_batch_plan(sl.h_enc, uint32_t(enc.size()));
                need[1] = dec.empty() ? 0 : rans_decode_batch_scratch_size(uint32_t(dec.size()));
                need[2] = up(sizeof(rans_encode_stream) * enc.size()) + up(sizeof(rans_stream) * dec.size());
                need[3] = up(8 * enc.size()) + up(4 * enc.size()) + up(4 * dec.size());
            };
            auto alloc_all = [&]() {
                for (int k = 0; k < 4; ++k) {
                    if (!s->arena.alloc(need[k], &offs[k])) {
                        for (int j = 0; j < k; ++j) s->arena.release(offs[j], need[j]);
                        return false;
                    }
                }
                return true;
            };
            auto give_back = [&](std::vector<Req> &v, size_t keep) {
                while (v.size() > keep) {
                    const Req q = v.back();
                    v.pop_back();
                    release_payload(q);
                    pending.push_front(q.id);
                }
            };
            plan_batch();
            bool ok = alloc_all();
            if (!ok && enc.size() + dec.size() > 1) {
                const uint32_t head = std::min(enc.empty() ? ~0u : enc.front().id,
                                               dec.empty() ? ~0u : dec.front().id);
                const bool head_enc = !enc.empty() && enc.front().id == head;
                give_back(enc, head_enc ? 1 : 0);
                give_back(dec, head_enc ? 0 : 1);
                std::sort(pending.begin(), pending.end());  // arrival order
                plan_batch();
                ok = alloc_all();
            }
            if (!ok) {
                const bool busy = std::any_of(s->slots.begin(), s->slots.end(),
                                              [](const Slot &x) { return x.phase != 0; });
                std::vector<Req> &v = enc.empty() ? dec : enc;
                if (!busy) {  // alone and nothing will free memory: it can never run
                    const Req q = v.front();
                    release_payload(q);
                    results[q.id].status = RANS_ERR_OOM;
                    results[q.id].admit_s = results[q.id].done_s = seconds_since(t0);
                    ++done;
                    v.clear();
                    progressed = true;
                } else {
                    give_back(v, 0);
                }
                break;
            }
            const uint64_t enc_scratch = need[0], dec_scratch = need[1];
            const uint64_t desc_bytes = need[2], res_bytes = need[3];
            const uint64_t o_es = offs[0], o_ds = offs[1], o_desc = offs[2], o_res = offs[3];
            sl.batch_allocs = {{o_es, enc_scratch}, {o_ds, dec_scratch}, {o_desc, desc_bytes}, {o_res, res_bytes}};
            sl.enc = std::move(enc);
            sl.dec = std::move(dec);
            sl.batch = batches++;
            progressed = true;
            const double t_admit = seconds_since(t0);
            for (const Req &q : sl.enc) results[q.id].admit_s = t_admit, results[q.id].batch = sl.batch;
            for (const Req &q : sl.dec) results[q.id].admit_s = t_admit, results[q.id].batch = sl.batch;
            for (size_t k = 0; k < sl.dec.size(); ++k) {
                const rans_request &r = reqs[sl.dec[k].id];
                rans_stream &d = sl.h_dec[k];
                d.msg = input_of(sl.dec[k]);
                d.msg_size = r.input_size;
                d.symbols = output_of(sl.dec[k]);
                d.n_symbols = r.n_symbols;
                d.table = r.table;
                d.n_lanes = r.n_lanes;
                d.chunk_symbols = r.chunk_symbols;
                d.reserved = 0;
            }
            uint8_t *desc_enc = s->d_arena + o_desc;
            uint8_t *desc_dec = desc_enc + up(sizeof(rans_encode_stream) * sl.enc.size());
            uint64_t *d_sizes = reinterpret_cast<uint64_t *>(s->d_arena + o_res);
            uint32_t *d_st_enc = reinterpret_cast<uint32_t *>(s->d_arena + o_res + up(8 * sl.enc.size()));
            uint32_t *d_st_dec = reinterpret_cast<uint32_t *>(reinterpret_cast<uint8_t *>(d_st_enc) +
                                                              up(4 * sl.enc.size()));
            cudaStream_t st = sl.stream;
            bool cu = true;
            for (const Req &q : sl.enc)
                cu = cu && (on_device(reqs[q.id]) ||
                            cudaMemcpyAsync(s->d_arena + q.in_off, reqs[q.id].input, q.in_len,
                                            cudaMemcpyHostToDevice, st) == cudaSuccess);
            for (const Req &q : sl.dec)
                cu = cu && (on_device(reqs[q.id]) ||
                            cudaMemcpyAsync(s->d_arena + q.in_off, reqs[q.id].input, q.in_len,
                                            cudaMemcpyHostToDevice, st) == cudaSuccess);
            if (!sl.enc.empty()) {
                cu = cu && cudaMemcpyAsync(desc_enc, sl.h_enc, sizeof(rans_encode_stream) * sl.enc.size(),
                                           cudaMemcpyHostToDevice, st) == cudaSuccess;
                cu = cu && rans_encode_batch(reinterpret_cast<rans_encode_stream *>(desc_enc),
                                             uint32_t(sl.enc.size()), s->d_freqs, s->n_tables, d_sizes,
                                             d_st_enc, s->d_arena + o_es, enc_scratch,
                                             reinterpret_cast<rans_stream_t>(st)) == RANS_OK;
                cu = cu && cudaMemcpyAsync(sl.h_sizes, d_sizes, 8 * sl.enc.size(),
                                           cudaMemcpyDeviceToHost, st) == cudaSuccess;
                cu = cu && cudaMemcpyAsync(sl.h_status, d_st_enc, 4 * sl.enc.size(),
                                           cudaMemcpyDeviceToHost, st) == cudaSuccess;
            }
            if (!sl.dec.empty()) {
                cu = cu && cudaMemcpyAsync(desc_dec, sl.h_dec, sizeof(rans_stream) * sl.dec.size(),
                                           cudaMemcpyHostToDevice, st) == cudaSuccess;
                cu = cu && rans_decode_batch(reinterpret_cast<rans_stream *>(desc_dec),
                                             uint32_t(sl.dec.size()), s->d_freqs, s->n_tables, d_st_dec,
                                             s->d_arena + o_ds, dec_scratch,
                                             reinterpret_cast<rans_stream_t>(st)) == RANS_OK;
                cu = cu && cudaMemcpyAsync(sl.h_status + s->max_batch, d_st_dec, 4 * sl.dec.size(),
                                           cudaMemcpyDeviceToHost, st) == cudaSuccess;
                for (const Req &q : sl.dec)
                    cu = cu && (on_device(reqs[q.id]) ||
                                cudaMemcpyAsync(reqs[q.id].output, s->d_arena + q.out_off,
                                                q.out_len, cudaMemcpyDeviceToHost,
                                                st) == cudaSuccess);
            }
            cu = cu && cudaEventRecord(sl.ev, st) == cudaSuccess;
            if (!cu) rc = RANS_ERR_CUDA;
            sl.phase = 1;
        }

        if (!progressed) {
            // nothing to do until the next arrival or completion
            const bool busy = std::any_of(s->slots.begin(), s->slots.end(),
                                          [](const Slot &x) { return x.phase != 0; });
            if (!busy && next < n) {
                const double wait = reqs[next].arrival_s - seconds_since(t0);
                if (wait > 200e-6) std::this_thread::sleep_for(std::chrono::duration<double>(wait - 100e-6));
            } else {
                std::this_thread::sleep_for(std::chrono::microseconds(5));
            }
        }
    }
    if (rc != RANS_OK) {
        for (Slot &sl : s->slots) cudaStreamSynchronize(sl.stream);
    }
    return rc;
}
