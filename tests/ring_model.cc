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
// Two consumer disciplines:
//  fifo    one token at a time at the ring's head; capacity >= the worker's
//          segments;
//  window  the batched kernel's: the first kWindow positions are read, up
//          to B ready ones are taken (B = 16, the kernel's batch when a row
//          is one 16-byte chunk per lane; mode window8: B = 8, its batch for
//          wider rows; a position reserved but not yet written does not hold
//          back the ones behind it), the head moves past the taken prefix,
//          the batch's long visits (a fixed quarter of the segments, as the
//          kernel's visits of >= 32 ratings) run first and each is handed on
//          right after its visit, and the other tokens are handed on
//          together at the end of the batch; capacity >= segments +
//          kWindow + 1.  The
//          tokens of urgent items (at least half the segments of the
//          item with most) travel through a second ring per worker
//          (capacity >= urgent items + 1), taken one at a time before each
//          batch and before each visit of a batch, and handed on at once.
// Every slot also records the lap last taken from it (model instrumentation
// only), so a producer that would overwrite a token not yet taken is seen.
//
// usage: ring_model <p> <n_items> <max_deg> <epochs> <seed> <fault> [mode]
//   fault: none | drop (one token never sent) | dup (one token sent twice)
//          | stall (one worker sleeps between visits)
//          | slowpub (some producers pause between reserving and writing)
//          | smallring (rings of a quarter of the segments: a planted mistake)
//   mode:  fifo (default) | window | window8
// prints: status=<ok|timeout|ownership|overwrite> visits=<v> expected=<S*E>
//         exact_once=<0|1> per_item_epochs_ok=<0|1> urgent_items=<u>
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

constexpr int kWindow = 16;

struct Model {
  int p = 0, n = 0, epochs = 0;
  uint64_t seed = 0;
  std::string fault;
  bool window = false;
  int batch = 16;  // tokens taken at once (window disciplines)
  // layout: segments per item, each with a worker
  std::vector<int> seg_worker, seg_item;
  std::vector<std::vector<int>> item_segs;    // segments of item j
  std::vector<int> nseg;                       // per worker
  // rings
  std::vector<int> log2cap;
  std::vector<int64_t> base;
  std::vector<std::atomic<uint64_t>> slots;
  std::vector<std::atomic<uint32_t>> taken_lap;  // per slot: lap last taken (~0: none)
  // urgent rings (window discipline only): p rings of 2^lgu slots
  std::vector<char> urgent;
  int lgu = 5;
  std::vector<std::atomic<uint64_t>> uslots;
  std::vector<std::atomic<uint32_t>> utail;
  std::vector<std::atomic<uint32_t>> utaken_lap;
  std::vector<std::atomic<uint32_t>> tail;
  // token state (owned by the holder)
  std::vector<int> hop, epoch;
  std::vector<std::vector<int>> order;         // current epoch's order per item
  std::vector<std::atomic<int>> owner;
  std::vector<std::atomic<int>> visits;        // per (segment, epoch)
  std::atomic<int> status{0};  // 0 ok, 1 timeout, 2 ownership, 3 overwrite
  std::atomic<uint32_t> pushes{0};
  std::atomic<int64_t> total{0};

  Model(int p_, int n_, int maxdeg, int e_, uint64_t s_, std::string f, bool win, int b_)
      : p(p_), n(n_), epochs(e_), seed(s_), fault(std::move(f)), window(win), batch(b_),
        slots(0), taken_lap(0), uslots(0), utail(p_), utaken_lap(0), tail(p_), owner(n_),
        visits(0) {
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
      int need = window ? nseg[q] + kWindow + 1 : nseg[q];
      if (fault == "smallring") need = nseg[q] / 4;
      int lg = 0;
      while ((1 << lg) < need || lg < 1) ++lg;
      log2cap[q] = lg;
      base[q] = b;
      b += int64_t(1) << lg;
    }
    base[p] = b;
    std::vector<std::atomic<uint64_t>> s(b);
    slots.swap(s);
    for (auto& x : slots) x.store(~0ull);
    std::vector<std::atomic<uint32_t>> tl(b);
    taken_lap.swap(tl);
    for (auto& x : taken_lap) x.store(~0u);
    size_t maxd = 0;
    for (auto& v : item_segs) maxd = std::max(maxd, v.size());
    urgent.assign(n, 0);
    int n_urgent = 0;
    for (int j = 0; j < n; ++j)
      if (window && 2 * item_segs[j].size() >= maxd) {
        urgent[j] = 1;
        ++n_urgent;
      }
    int need_u = n_urgent + 1;
    if (fault == "smallring") need_u = std::max(1, n_urgent / 4);
    while ((1 << lgu) < need_u) ++lgu;
    std::vector<std::atomic<uint64_t>> us(size_t(p) << lgu);
    uslots.swap(us);
    for (auto& x : uslots) x.store(~0ull);
    std::vector<std::atomic<uint32_t>> utl(size_t(p) << lgu);
    utaken_lap.swap(utl);
    for (auto& x : utaken_lap) x.store(~0u);
    for (auto& t : utail) t.store(0);
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
    const bool u = urgent[seg_item[seg]] != 0;
    const uint32_t pos = (u ? utail[q] : tail[q]).fetch_add(1, std::memory_order_relaxed);
    const int lg = u ? lgu : log2cap[q];
    const int64_t at = (u ? (int64_t(q) << lgu) : base[q]) + (pos & ((1u << lg) - 1u));
    auto& tlap = u ? utaken_lap[at] : taken_lap[at];
    auto& slot = u ? uslots[at] : slots[at];
    if (fault == "slowpub" && pushes.fetch_add(1) % 5 == 0)
      std::this_thread::sleep_for(std::chrono::microseconds(150));
    // the slot's previous lap must have been taken before it is written again
    const uint32_t lap = pos >> lg;
    if (lap > 0 && tlap.load(std::memory_order_acquire) != lap - 1) {
      int z = 0;
      status.compare_exchange_strong(z, 3);
    }
    slot.store((uint64_t(lap) << 32) | uint32_t(seg), std::memory_order_release);
  }

  int pop(int q, uint32_t head) {
    const int lg = log2cap[q];
    auto& slot = slots[base[q] + (head & ((1u << lg) - 1u))];
    const uint32_t lap = head >> lg;
    const auto t0 = std::chrono::steady_clock::now();
    for (uint64_t it = 0; it < (1ull << 28); ++it) {
      const uint64_t v = slot.load(std::memory_order_acquire);
      if (uint32_t(v >> 32) == lap) {
        taken_lap[base[q] + (head & ((1u << lg) - 1u))].store(lap, std::memory_order_release);
        return int(uint32_t(v));
      }
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

  // One visit of segment seg by worker q: ownership check, accounting, the
  // token's next hop.  Returns the next segment, or -1 after its last epoch.
  int visit(int q, int seg) {
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
    return ne < epochs ? order[j][nh] : -1;
  }

  // The batched kernel's discipline (see the header comment).
  void worker_window(int q) {
    const int64_t quota = int64_t(nseg[q]) * epochs;
    const int lg = log2cap[q];
    const uint32_t mask = (1u << lg) - 1u;
    uint32_t head = 0, taken = 0, head_u = 0;
    int64_t done = 0;
    auto t_last = std::chrono::steady_clock::now();
    // an urgent token waiting at the head of the urgent ring: visited and
    // handed on at once
    auto try_urgent = [&]() -> bool {
      const int64_t at = (int64_t(q) << lgu) + (head_u & ((1u << lgu) - 1u));
      const uint64_t v = uslots[at].load(std::memory_order_acquire);
      if (uint32_t(v >> 32) != (head_u >> lgu)) return false;
      utaken_lap[at].store(head_u >> lgu, std::memory_order_release);
      ++head_u;
      ++done;
      const int nx = visit(q, int(uint32_t(v)));
      if (nx >= 0) push(seg_worker[nx], nx);
      t_last = std::chrono::steady_clock::now();
      return true;
    };
    while (done < quota) {
      while (done < quota && try_urgent()) {
      }
      if (done >= quota) break;
      int got[kWindow];
      uint32_t ready = 0;
      for (int i = 0; i < kWindow; ++i) {
        if ((taken >> i) & 1u) continue;
        const uint32_t pos = head + uint32_t(i);
        const uint64_t v = slots[base[q] + (pos & mask)].load(std::memory_order_acquire);
        if (uint32_t(v >> 32) == (pos >> lg)) {
          ready |= 1u << i;
          got[i] = int(uint32_t(v));
        }
      }
      if (!ready) {
        if (status.load(std::memory_order_relaxed) != 0) return;
        if (std::chrono::steady_clock::now() - t_last > std::chrono::milliseconds(300)) {
          int z = 0;
          status.compare_exchange_strong(z, 1);
          return;
        }
        std::this_thread::yield();
        continue;
      }
      t_last = std::chrono::steady_clock::now();
      std::vector<int> longv, shortv;
      int taken_now = 0;
      for (int i = 0; i < kWindow && taken_now < batch; ++i) {
        if (!((ready >> i) & 1u)) continue;
        const uint32_t pos = head + uint32_t(i);
        taken_lap[base[q] + (pos & mask)].store(pos >> lg, std::memory_order_release);
        taken |= 1u << i;
        (is_long(got[i]) ? longv : shortv).push_back(got[i]);
        ++taken_now;
      }
      while (taken & 1u) {  // the head moves past the taken prefix
        taken >>= 1;
        ++head;
      }
      done += int64_t(taken_now);
      for (int seg : longv) {  // long visits first, each handed on at once
        while (try_urgent()) {
        }
        const int nx = visit(q, seg);
        if (nx >= 0) push(seg_worker[nx], nx);
      }
      std::vector<int> next;
      for (int seg : shortv) {
        while (try_urgent()) {
        }
        next.push_back(visit(q, seg));
      }
      for (int nseg_id : next)  // handed on together at the end of the batch
        if (nseg_id >= 0) push(seg_worker[nseg_id], nseg_id);
    }
  }

  // a fixed quarter of the segments stand for the kernel's long visits
  static bool is_long(int seg) { return ((uint32_t(seg) * 2654435761u) >> 30) == 0; }

  void worker(int q) {
    if (window) {
      worker_window(q);
      return;
    }
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
      shuffle_order(j, 0);  // (push() routes urgent items to the urgent rings)
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
  if (argc != 7 && argc != 8) {
    std::fprintf(stderr, "usage: ring_model p n maxdeg epochs seed fault [fifo|window|window8]\n");
    return 2;
  }
  const std::string mode = argc == 8 ? argv[7] : "fifo";
  const bool window = mode == "window" || mode == "window8";
  Model M(std::atoi(argv[1]), std::atoi(argv[2]), std::atoi(argv[3]), std::atoi(argv[4]),
          std::strtoull(argv[5], nullptr, 10), argv[6], window, mode == "window8" ? 8 : 16);
  M.run();
  const int64_t S = int64_t(M.seg_worker.size());
  bool exact = true;
  for (auto& v : M.visits)
    if (v.load() != 1) exact = false;
  bool per_item = true;
  for (int j = 0; j < M.n; ++j)
    if (M.epoch[j] != M.epochs || M.hop[j] != 0) per_item = false;
  const char* st = M.status == 0   ? "ok"
                   : M.status == 1 ? "timeout"
                   : M.status == 2 ? "ownership"
                                   : "overwrite";
  int n_urgent = 0;
  for (char u : M.urgent) n_urgent += u;
  std::printf(
      "status=%s visits=%lld expected=%lld exact_once=%d per_item_epochs_ok=%d urgent_items=%d\n",
      st, (long long)M.total.load(), (long long)(S * M.epochs), exact ? 1 : 0, per_item ? 1 : 0,
      n_urgent);
  return 0;
}
