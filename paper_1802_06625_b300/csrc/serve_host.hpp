// Host side of the request loop (prune_server_*): the device-memory arena
// that admission draws on, the layout of one stream's resident state, and
// the planner that decides which streams advance in a step.  Plain C++ with
// no CUDA dependency, so the CPU tests compile and exercise it directly.
//
// The model follows the paper's runtime view (Sec. IV-V): every admitted
// stream is one instance of the canonical graph with its own FIFOs and delay
// token; instances are independent DPGs, so one step fires the next frames of
// many streams together, and a stream whose sink FIFO (its result ring) is
// full does not fire (the FIFO-space firing condition).
#pragma once
#include <algorithm>
#include <cstdint>
#include <deque>
#include <map>
#include <vector>

namespace prune {

// First-fit sub-allocator over offsets [0, size) with coalescing of freed
// neighbours.  Every block starts on an `align` boundary and its size is
// rounded up to one.
class Arena {
 public:
  explicit Arena(uint64_t size = 0, uint64_t align = 256) { reset(size, align); }

  void reset(uint64_t size, uint64_t align = 256) {
    align_ = align;
    size_ = size / align * align;
    free_.clear();
    live_.clear();
    used_ = 0;
    if (size_) free_[0] = size_;
  }

  // false (and nothing changed) when no free hole holds `bytes`
  bool alloc(uint64_t bytes, uint64_t *off) {
    const uint64_t need = std::max<uint64_t>(align_, (bytes + align_ - 1) / align_ * align_);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < need) continue;
      const uint64_t o = it->first, rest = it->second - need;
      free_.erase(it);
      if (rest) free_[o + need] = rest;
      live_[o] = need;
      used_ += need;
      *off = o;
      return true;
    }
    return false;
  }

  // false when `off` is not the start of a live block
  bool release(uint64_t off) {
    auto it = live_.find(off);
    if (it == live_.end()) return false;
    uint64_t o = off, n = it->second;
    live_.erase(it);
    used_ -= n;
    auto nx = free_.lower_bound(o);
    if (nx != free_.end() && nx->first == o + n) {  // merge the hole after
      n += nx->second;
      nx = free_.erase(nx);
    }
    if (nx != free_.begin()) {                      // merge the hole before
      auto pv = std::prev(nx);
      if (pv->first + pv->second == o) {
        o = pv->first;
        n += pv->second;
        free_.erase(pv);
      }
    }
    free_[o] = n;
    return true;
  }

  uint64_t size() const { return size_; }
  uint64_t used() const { return used_; }
  uint64_t largest_free() const {
    uint64_t m = 0;
    for (auto &f : free_) m = std::max(m, f.second);
    return m;
  }
  size_t holes() const { return free_.size(); }
  size_t blocks() const { return live_.size(); }

 private:
  uint64_t align_ = 256, size_ = 0, used_ = 0;
  std::map<uint64_t, uint64_t> free_;  // offset -> bytes
  std::map<uint64_t, uint64_t> live_;  // offset -> bytes
};

// Byte offsets of one stream's resident state inside its arena block, each
// 256-byte aligned: taps [T], H [N*N] and its tensor-core operands, the
// double-buffered delay token [2][T-1], the FIR output and block energies of
// the frames it fires in one step, and the result ring of `ring` frames
// (c, idx, compacted HX output).
struct StreamLayout {
  uint64_t taps, H, bops, fops, hist, y, energy, c, idx, out, total;
};

inline uint64_t align_up(uint64_t v, uint64_t a) { return (v + a - 1) / a * a; }

inline StreamLayout stream_layout(int64_t F, int64_t B, int64_t T, int64_t N, int64_t fps, int64_t ring,
                                  uint64_t bops_bytes, uint64_t fops_bytes = 0) {
  StreamLayout l{};
  uint64_t o = 0;
  auto take = [&](uint64_t bytes) {
    const uint64_t at = o;
    o = align_up(o + std::max<uint64_t>(bytes, 1), 256);
    return at;
  };
  const uint64_t L = static_cast<uint64_t>(F) * B;
  l.taps = take(8 * static_cast<uint64_t>(T));
  l.H = take(8 * static_cast<uint64_t>(N) * N);
  l.bops = take(bops_bytes);
  l.fops = take(fops_bytes);
  l.hist = take(8 * 2 * static_cast<uint64_t>(std::max<int64_t>(T - 1, 1)));
  l.y = take(8 * L * fps);
  l.energy = take(4 * static_cast<uint64_t>(F) * fps);
  l.c = take(4 * static_cast<uint64_t>(ring));
  l.idx = take(4 * static_cast<uint64_t>(F) * ring);
  l.out = take(8 * L * ring);
  l.total = o;
  return l;
}

// Frames queued by the caller: frame q of the segment is at x + (q % period) * F*B.
struct Segment {
  const void *x;
  int64_t n, period, next;  // next: frames of this segment already fired
};

struct StreamState {
  int64_t id = 0;
  int32_t F = 0, T = 0;
  float tau = 0.f;
  int32_t s_taps = 0, s_h = 0;   // exponents of the scaled tensor-core operands
  uint64_t mem = 0, bytes = 0;   // arena block
  std::deque<Segment> queue;
  int64_t queued = 0;            // frames submitted and not yet fired
  int64_t fired = 0;             // frames enqueued on the device
  int64_t done = 0;              // frames whose step has completed
  int64_t pulled = 0;            // frames handed back from the result ring
  int32_t parity = 0;            // which half of the delay-token buffer holds the current token
  bool closing = false;
  int64_t last_step = -1;        // last step that fires this stream
};

// One frame of one stream in a step.  `prev` is the input of the frame
// before it when that frame fires in the same step (its last T-1 samples are
// this frame's delay token), else nullptr (the token is the resident one).
struct PlanEntry {
  int32_t stream;    // index into the stream table
  int64_t frame;     // frame number within the stream
  const void *x;     // the frame's input
  const void *prev;  // the previous frame's input within this step, or nullptr
  bool last;         // last frame of the stream in this step (writes the delay token)
};

// Which frames fire in the next step: every open stream, in admission order,
// advances by up to `fps` frames, as far as its queue and its free result
// slots allow, up to `max_entries` entries in all.  Consumes the frames from
// the queues and advances `fired`; the caller launches the entries.  B is
// the common block size (a frame of stream s is F_s * B complex64 samples).
inline std::vector<PlanEntry> plan_step(std::vector<StreamState> &streams, const std::vector<int32_t> &order,
                                        int32_t B, int32_t fps, int32_t ring, int32_t max_entries) {
  std::vector<PlanEntry> plan;
  for (int32_t si : order) {
    if (static_cast<int32_t>(plan.size()) >= max_entries) break;
    StreamState &s = streams[si];
    if (s.closing || s.queued == 0) continue;
    const int64_t space = ring - (s.fired - s.pulled);
    const int64_t room = static_cast<int64_t>(max_entries) - static_cast<int64_t>(plan.size());
    const int64_t k = std::min<int64_t>({static_cast<int64_t>(fps), s.queued, space, room});
    if (k <= 0) continue;
    const int64_t frame_bytes = static_cast<int64_t>(s.F) * B * 8;
    const void *prev = nullptr;
    for (int64_t j = 0; j < k; ++j) {
      Segment &g = s.queue.front();
      const void *x = static_cast<const char *>(g.x) + (g.next % g.period) * frame_bytes;
      plan.push_back(PlanEntry{si, s.fired + j, x, prev, j == k - 1});
      prev = x;
      if (++g.next == g.n) s.queue.pop_front();
    }
    s.queued -= k;
    s.fired += k;
  }
  return plan;
}

}  // namespace prune
