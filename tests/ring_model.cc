// ring_model.cc -- host-thread model of the token-passing protocol of the
// persistent NOMAD kernel, for testing the protocol logic and its failure
// detection on the CPU (no GPU involved).
//
// p worker threads; worker q owns a ring of lap-tagged 64-bit slots
// {lap:32 | segment:32} with capacity >= the number of items it holds.  A
// producer reserves a position with fetch_add on the ring's tail and
// publishes with a release store; the consumer alone advances its head and
// waits (bounded) until the slot shows the lap it expects.  Items circulate
// in epoch mode: in every epoch item j visits each of its segments once, in
// a fresh random order (Sec. 3.4's permutation circulation).  Every wait is
// bounded; a worker that gives up raises the shared status word.
//
// usage: ring_model <p> <n_items> <max_deg> <epochs> <seed> <fault>
//   fault: none | drop (one token never sent) | dup (one token sent twice)
//          | stall (one worker sleeps between visits)
// prints: status=<ok|timeout|ownership> visits=<v> expected=<S*E>
//         exact_once=<0|1> per_item_epochs_ok=<0|1>
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <string>
#include <thread>
#include <vector>

namespace {

struct Model {
  int p = 0, n = 0, epochs = 0;
  uint64_t seed = 0;
  std::string fault;
  // layout: segments per item, each with a worker
  std::vector<int> seg_worker, seg_item;
  std::vector<std::vector<int>> item_segs;    // segments of item j
  std::vector<int> nseg;                       // per worker
  // rings
  std::vector<int> log2cap;
  std::vector<int64_t> base;
  std::vector<std::atomic<uint64_t>> slots;
  std::vector<std::atomic<uint32_t>> tail;
  // token state (owned by the holder)
  std::vector<int> hop, epoch;
  std::vector<std::vector<int>> order;         // current epoch's order per item
  std::vector<std::atomic<int>> owner;
  std::vector<std::atomic<int>> visits;        // per (segment, epoch)
  std::atomic<int> status{0};                  // 0 ok, 1 timeout, 2 ownership
  std::atomic<int64_t> total{0};

  Model(int p_, int n_, int maxdeg, int e_, uint64_t s_, std::string f)
      : p(p_), n(n_), epochs(e_), seed(s_), fault(std::move(f)),
        slots(0), tail(p_), owner(n_), visits(0) {
    std::mt19937_64 rng(seed);
    item_segs.resize(n);
    nseg.assign(p, 0);
    for (int j = 0; j < n; ++j) {
      const int d = 1 + int(rng() % uint64_t(maxdeg < p ? maxdeg : p));
      std::vector<int> ws(p);
      for (int q = 0; q < p; ++q) ws[q] = q;
      std::shuffle(ws.begin(), ws.end(), rng);
      for (int t = 0; t < d; ++t) {
        item_segs[j].push_back(int(seg_worker.size()));
        seg_worker.push_back(ws[t]);
        seg_item.push_back(j);
        nseg[ws[t]]++;
      }
    }
    log2cap.resize(p);
    base.resize(p + 1);
    int64_t b = 0;
    for (int q = 0; q < p; ++q) {
      int lg = 0;
      while ((1 << lg) < nseg[q] || lg < 1) ++lg;
      log2cap[q] = lg;
      base[q] = b;
      b += int64_t(1) << lg;
    }
    base[p] = b;
    std::vector<std::atomic<uint64_t>> s(b);
    slots.swap(s);
    for (auto& x : slots) x.store(~0ull);
    for (auto& t : tail) t.store(0);
    hop.assign(n, 0);
    epoch.assign(n, 0);
    order.resize(n);
    for (auto& o : owner) o.store(-1);
    std::vector<std::atomic<int>> v(seg_worker.size() * size_t(epochs));
    visits.swap(v);
    for (auto& x : visits) x.store(0);
  }

  void shuffle_order(int j, int e) {
    order[j] = item_segs[j];
    std::mt19937_64 rng(seed * 1000003ull + uint64_t(j) * 7919ull + uint64_t(e));
    std::shuffle(order[j].begin(), order[j].end(), rng);
  }

  void push(int q, int seg) {
    const uint32_t pos = tail[q].fetch_add(1, std::memory_order_relaxed);
    const int lg = log2cap[q];
    auto& slot = slots[base[q] + (pos & ((1u << lg) - 1u))];
    slot.store((uint64_t(pos >> lg) << 32) | uint32_t(seg), std::memory_order_release);
  }

  int pop(int q, uint32_t head) {
    const int lg = log2cap[q];
    auto& slot = slots[base[q] + (head & ((1u << lg) - 1u))];
    const uint32_t lap = head >> lg;
    const auto t0 = std::chrono::steady_clock::now();
    for (uint64_t it = 0; it < (1ull << 28); ++it) {
      const uint64_t v = slot.load(std::memory_order_acquire);
      if (uint32_t(v >> 32) == lap) return int(uint32_t(v));
      if ((it & 255) == 255) {
        if (status.load(std::memory_order_relaxed) != 0) return -1;
        if (std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(300)) break;
        std::this_thread::yield();
      }
    }
    int z = 0;
    status.compare_exchange_strong(z, 1);
    return -1;
  }

  void worker(int q) {
    const int64_t quota = int64_t(nseg[q]) * epochs;
    uint32_t head = 0;
    for (int64_t v = 0; v < quota; ++v, ++head) {
      const int seg = pop(q, head);
      if (seg < 0) return;
      const int j = seg_item[seg];
      if (owner[j].exchange(q) != -1) {
        int z = 0;
        status.compare_exchange_strong(z, 2);
      }
      const int e = epoch[j];
      if (e >= 0 && e < epochs) visits[size_t(seg) * epochs + e].fetch_add(1);
      total.fetch_add(1);
      if (fault == "stall" && q == 0)
        std::this_thread::sleep_for(std::chrono::microseconds(200));
      int nh = hop[j] + 1, ne = e;
      if (nh == int(item_segs[j].size())) {
        nh = 0;
        ne = e + 1;
        if (ne < epochs) shuffle_order(j, ne);
      }
      hop[j] = nh;
      epoch[j] = ne;
      if (owner[j].exchange(-1) != q) {
        int z = 0;
        status.compare_exchange_strong(z, 2);
      }
      if (ne < epochs) {
        const int nseg_id = order[j][nh];
        push(seg_worker[nseg_id], nseg_id);
      }
    }
  }

  void run() {
    for (int j = 0; j < n; ++j) {
      shuffle_order(j, 0);
      if (fault == "drop" && j == 0) continue;
      push(seg_worker[order[j][0]], order[j][0]);
      if (fault == "dup" && j == 0) push(seg_worker[order[j][0]], order[j][0]);
    }
    std::vector<std::thread> th;
    for (int q = 0; q < p; ++q) th.emplace_back(&Model::worker, this, q);
    for (auto& t : th) t.join();
  }
};

}  // namespace

int main(int argc, char** argv) {
  if (argc != 7) {
    std::fprintf(stderr, "usage: ring_model p n maxdeg epochs seed fault\n");
    return 2;
  }
  Model M(std::atoi(argv[1]), std::atoi(argv[2]), std::atoi(argv[3]), std::atoi(argv[4]),
          std::strtoull(argv[5], nullptr, 10), argv[6]);
  M.run();
  const int64_t S = int64_t(M.seg_worker.size());
  bool exact = true;
  for (auto& v : M.visits)
    if (v.load() != 1) exact = false;
  bool per_item = true;
  for (int j = 0; j < M.n; ++j)
    if (M.epoch[j] != M.epochs || M.hop[j] != 0) per_item = false;
  const char* st = M.status == 0 ? "ok" : (M.status == 1 ? "timeout" : "ownership");
  std::printf("status=%s visits=%lld expected=%lld exact_once=%d per_item_epochs_ok=%d\n", st,
              (long long)M.total.load(), (long long)(S * M.epochs), exact ? 1 : 0,
              per_item ? 1 : 0);
  return 0;
}
