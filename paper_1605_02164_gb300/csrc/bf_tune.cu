// Tuning table: measured tile heights of the windowed kernels.
//
// The tile height of the fused kernels (output rows per CTA tile, a multiple
// of 16) does not change any pixel's arithmetic, only how the work spreads
// over the SMs and how much halo each tile recomputes.  Without an entry the
// launches use their cost models (waves of tiles x steps per tile for an image
// alone, the tallest tile in a batch).  The autotuner (tune.py) times the
// candidate heights per (variant, d, radius class, size class, context) and
// stores the fastest here; every launch consults the table first.  The radius
// class ceil(r / 8) groups the radii that share the tensor-core tile geometry
// (the row lag of the vertical window and the tallest tile).
#include <math.h>

#include <map>
#include <mutex>
#include <tuple>

#include "bf_internal.cuh"

namespace bf {
namespace {

using Key = std::tuple<int, int, int, int, int>;  // variant, d, radius class, size class, context
std::mutex g_tune_mu;
std::map<Key, int> g_tune;

int radius_class(int r) { return (r + 7) / 8; }

int size_class_of(int H, int W) {
    const int ch = (int)floor(2.0 * log2((double)(H > 0 ? H : 1)));
    const int cw = (int)floor(2.0 * log2((double)(W > 0 ? W : 1)));
    return 32 * ch + cw;
}

bool valid_key(int variant, int d, int r, int context) {
    return (variant == BF_FP32 || variant == BF_FP16TC || variant == BF_BF16TC) && d >= 1 && d <= BF_MAX_D &&
           r >= 0 && r <= BF_MAX_RADIUS && (context == BF_TUNE_ALONE || context == BF_TUNE_BATCH);
}

}  // namespace

int tune_rows(int variant, int d, int r, int H, int W, int context) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (g_tune.empty()) return 0;
    const auto it = g_tune.find(Key{variant, d, radius_class(r), size_class_of(H, W), context});
    return it == g_tune.end() ? 0 : it->second;
}

}  // namespace bf

extern "C" int bf_tune_size_class(int H, int W) {
    if (H <= 0 || W <= 0) return BF_ERR_ARG;
    return bf::size_class_of(H, W);
}

extern "C" int bf_tune_set(int variant, int d, int r, int size_class, int context, int tile_rows) {
    if (!bf::valid_key(variant, d, r, context) || size_class < 0) return BF_ERR_ARG;
    if (tile_rows < 0 || tile_rows > 128 || tile_rows % 16 != 0) return BF_ERR_ARG;
    std::lock_guard<std::mutex> lk(bf::g_tune_mu);
    const bf::Key k{variant, d, bf::radius_class(r), size_class, context};
    if (tile_rows == 0)
        bf::g_tune.erase(k);
    else
        bf::g_tune[k] = tile_rows;
    return BF_OK;
}

extern "C" int bf_tune_get(int variant, int d, int r, int size_class, int context, int *tile_rows) {
    if (!tile_rows || !bf::valid_key(variant, d, r, context) || size_class < 0) return BF_ERR_ARG;
    std::lock_guard<std::mutex> lk(bf::g_tune_mu);
    const auto it = bf::g_tune.find(bf::Key{variant, d, bf::radius_class(r), size_class, context});
    *tile_rows = it == bf::g_tune.end() ? 0 : it->second;
    return BF_OK;
}

extern "C" int bf_tune_clear(void) {
    std::lock_guard<std::mutex> lk(bf::g_tune_mu);
    bf::g_tune.clear();
    return BF_OK;
}

extern "C" int bf_tune_count(void) {
    std::lock_guard<std::mutex> lk(bf::g_tune_mu);
    return (int)bf::g_tune.size();
}
