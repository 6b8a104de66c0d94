// transforms.cu -- process-wide state of the transform launchers: the
// tile-shape table the autotuner records, the shape it forces while timing,
// and the flag of a launch with no kernel for its (type, mode) pair.  The
// kernels and launchers are in transforms.cuh, instantiated per arithmetic
// type in transforms_f64.cu, transforms_f32.cu and transforms_df_a.cu, _b.cu and _c.cu.
#include <atomic>

#include "transforms.cuh"

namespace rsfde {

static int g_tuned[TK_COUNT][16][2];
static thread_local int g_force_groups = 0;
static std::atomic<int> g_unsupported{0};

void tune_force_groups(int F) { g_force_groups = F; }
int tune_forced() { return g_force_groups; }
void tune_record(int kind, int log2L, int wide, int F) {
  if (kind >= 0 && kind < TK_COUNT && log2L >= 0 && log2L < 16) g_tuned[kind][log2L][wide ? 1 : 0] = F;
}
int tune_lookup(int kind, int log2L, int wide) {
  return (kind >= 0 && kind < TK_COUNT && log2L >= 0 && log2L < 16) ? g_tuned[kind][log2L][wide ? 1 : 0] : 0;
}
void note_unsupported_launch() { g_unsupported.store(1); }
bool take_unsupported_launch() { return g_unsupported.exchange(0) != 0; }

template int max_groups<double>(int, int);
template int max_groups<float>(int, int);
template int max_groups<df>(int, int);

}  // namespace rsfde
