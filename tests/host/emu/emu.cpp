// Launch machinery of the host emulation (see cuda_runtime.h): the threads
// of a block are ucontext fibers of the calling host thread (all state is
// per host thread, so launches from several host threads are independent).
#include <setjmp.h>
#include <ucontext.h>

#include <cstdio>
#include <vector>

#include "cuda_runtime.h"

thread_local uint3 threadIdx;
thread_local uint3 blockIdx;
thread_local dim3 blockDim;
thread_local dim3 gridDim;
thread_local EmuBarrier emu_block_bar;
thread_local EmuBarrier emu_warp_bar[32];
thread_local uint64_t emu_slot[32][32];
thread_local int emu_acc;
thread_local EmuBarrier emu_named_bar[16];
thread_local unsigned long long emu_ops;
thread_local unsigned long long emu_block_barriers;

namespace {
// A fiber starts on its own stack through setcontext (once); afterwards the
// fibers and the scheduler switch with _setjmp/_longjmp, which, unlike
// swapcontext, make no signal-mask system call.
struct Fiber {
  ucontext_t ctx;
  jmp_buf jb;
  bool started;
  const long* wait_on;  // generation counter this fiber waits to change
  long wait_gen;
  bool done;
};
thread_local jmp_buf g_sched;
thread_local std::vector<Fiber> g_fibers;
thread_local int g_cur;
thread_local const std::function<void()>* g_body;
constexpr size_t kStack = 256 * 1024;
// order in which a pass resumes the runnable threads: 0 ascending, 1
// descending, 2 a fresh pseudo-random permutation every pass.  A kernel
// without data races (every read of another thread's write separated from it
// by a barrier) gives the same results in every order.
int g_order = 0;
uint64_t g_seed = 1;

uint64_t next_rand() {  // xorshift64
  g_seed ^= g_seed << 13;
  g_seed ^= g_seed >> 7;
  g_seed ^= g_seed << 17;
  return g_seed;
}

void fiber_entry() {
  (*g_body)();
  g_fibers[g_cur].done = true;
  _longjmp(g_sched, 1);
}
}  // namespace

void emu_wait(EmuBarrier& b) {
  const long g = b.gen;
  if (++b.count == b.n) {
    b.count = 0;
    ++b.gen;
    if (&b == &emu_block_bar) ++emu_block_barriers;
    return;
  }
  Fiber& f = g_fibers[g_cur];
  f.wait_on = &b.gen;
  f.wait_gen = g;
  if (!_setjmp(f.jb)) _longjmp(g_sched, 1);
}

void emu_launch(dim3 grid, dim3 block, const std::function<void()>& body) {
  const unsigned nt = block.x, nb = grid.x;
  if (nt == 0 || nb == 0) return;
  std::vector<std::vector<char>> stacks(nt, std::vector<char>(kStack));
  g_fibers.assign(nt, Fiber{});
  g_body = &body;
  blockDim = block;
  gridDim = grid;
  for (unsigned x = 0; x < nb; ++x) {
    blockIdx = uint3{x, 0, 0};
    emu_block_bar = EmuBarrier{0, 0, (int)nt};
    for (auto& nb16 : emu_named_bar) nb16 = EmuBarrier{0, 0, 64};
    for (unsigned w = 0; w < 32; ++w) {
      const int n = (w + 1) * 32 <= nt ? 32 : (w * 32 < nt ? (int)(nt - w * 32) : 0);
      emu_warp_bar[w] = EmuBarrier{0, 0, n};
    }
    for (unsigned t = 0; t < nt; ++t) {
      Fiber& f = g_fibers[t];
      f = Fiber{};
      getcontext(&f.ctx);
      f.ctx.uc_stack.ss_sp = stacks[t].data();
      f.ctx.uc_stack.ss_size = kStack;
      f.ctx.uc_link = nullptr;
      makecontext(&f.ctx, fiber_entry, 0);
    }
    unsigned alive = nt;
    std::vector<unsigned> order(nt);
    for (unsigned t = 0; t < nt; ++t) order[t] = g_order == 1 ? nt - 1 - t : t;
    while (alive > 0) {
      bool progress = false;
      if (g_order == 2)
        for (unsigned t = nt - 1; t > 0; --t) std::swap(order[t], order[next_rand() % (t + 1)]);
      for (unsigned o = 0; o < nt; ++o) {
        const unsigned t = order[o];
        Fiber& f = g_fibers[t];
        if (f.done || (f.wait_on && *f.wait_on == f.wait_gen)) continue;
        f.wait_on = nullptr;
        g_cur = (int)t;
        threadIdx = uint3{t, 0, 0};
        if (!_setjmp(g_sched)) {
          if (!f.started) {
            f.started = true;
            setcontext(&f.ctx);
          }
          _longjmp(f.jb, 1);
        }
        progress = true;
        if (f.done) --alive;
      }
      if (!progress) {
        std::fprintf(stderr, "emulation: block %u deadlocked (%u threads parked at a barrier)\n", x,
                     alive);
        std::abort();
      }
    }
  }
}

// the schedule of later launches (see g_order); seed for order 2
extern "C" void emu_set_schedule(int order, unsigned long long seed) {
  g_order = order;
  g_seed = seed ? seed : 1;
}
