// Host-side check of the tensor-core kernel's TMEM and shared-memory layout
// rules, for every MLP width, encoding width and depth the library accepts
// (built and run by tests/test_tc_layout.py; no GPU is touched).  For each
// variant: the accumulator regions (R0, the dW of every layer, dW_out where it
// is formed on the tensor cores) are disjoint and lie inside the columns the
// CTA allocates; that allocation is a power of two of at most 256 columns; the
// split form always forms dW_out on the tensor cores; and the CTAs per SM the
// launch bounds budget registers for fit the SM's shared memory and TMEM.
#include <cstdio>

#include "fused_tc.cuh"

using namespace prenom;

static int failures = 0;

#define CHECK(cond, ...)                                                                                              \
    do {                                                                                                              \
        if (!(cond)) {                                                                                                \
            std::printf("FAIL: " __VA_ARGS__);                                                                        \
            std::printf("\n");                                                                                        \
            ++failures;                                                                                               \
        }                                                                                                             \
    } while (0)

template <int W, int IN>
void check_variant()
{
    constexpr int INP = TcLayout<W, IN>::INP;
    const int R0 = tc_r0<W, IN>();
    CHECK(R0 >= W && R0 >= INP && R0 >= 16, "W%d IN%d: R0 %d too narrow", W, IN, R0);
    for (int split = 0; split < 2; ++split)
        for (int H = 1; H <= kMaxHidden; ++H) {
            const int cols = tc_cols<W, IN>(H, split != 0);
            CHECK(cols >= 32 && cols <= kTcCols && (cols & (cols - 1)) == 0, "W%d IN%d H%d split%d: %d columns", W,
                  IN, H, split, cols);
            // regions [begin, end) in allocation order
            int end = R0;
            const int dw0 = (int)dw_col<W, IN>(0);
            CHECK(dw0 == end, "W%d IN%d: dW_0 at %d, R0 ends at %d", W, IN, dw0, end);
            end = dw0 + INP;
            for (int l = 1; l < H; ++l) {
                const int dwl = (int)dw_col<W, IN>(l);
                CHECK(dwl >= end, "W%d IN%d H%d: dW_%d overlaps", W, IN, H, l);
                end = dwl + W;
            }
            const bool dwo = split && tc_dw_out<W, IN>(H);
            if (split)
                CHECK(dwo, "W%d IN%d H%d: the split form must form dW_out on the tensor cores", W, IN, H);
            if (dwo) {
                const int dwh = (int)dw_col<W, IN>(H);
                constexpr int dwo_cols = tc_dwo_transposed<W>() ? 16 : W;
                CHECK(dwh >= end, "W%d IN%d H%d: dW_out overlaps", W, IN, H);
                end = dwh + dwo_cols;
            }
            CHECK(end <= cols, "W%d IN%d H%d split%d: regions end at %d beyond %d columns", W, IN, H, split, end, cols);
            // the resident CTAs the registers are budgeted for fit TMEM and shared memory
            // (dynamic + 512 B static + 1 KB reserved per CTA of the SM's 228 KB)
            const int per_sm = split ? ((W <= 32) ? 3 : 2) : 2;
            const size_t smem = TcLayout<W, IN>::bytes(H, split != 0) + 512 + 1024;
            if (split && W <= 32 && H <= 2) {
                CHECK(per_sm * cols <= 512, "W%d IN%d H%d: %d CTAs need %d TMEM columns", W, IN, H, per_sm,
                      per_sm * cols);
                CHECK(per_sm * smem <= 228 * 1024, "W%d IN%d H%d: %d CTAs need %zu B of shared memory", W, IN, H,
                      per_sm, per_sm * smem);
            }
            CHECK(2 * cols <= 512 || per_sm == 1, "W%d IN%d H%d: two CTAs exceed TMEM", W, IN, H);
        }
}

int main()
{
    check_variant<16, 8>();
    check_variant<16, 16>();
    check_variant<16, 32>();
    check_variant<32, 8>();
    check_variant<32, 16>();
    check_variant<32, 32>();
    check_variant<64, 8>();
    check_variant<64, 16>();
    check_variant<64, 32>();
    if (failures == 0)
        std::printf("OK\n");
    return failures == 0 ? 0 : 1;
}
