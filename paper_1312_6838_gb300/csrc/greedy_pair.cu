// The persistent greedy kernel (greedy.cu) in its second CTA shape: 256
// threads with two CTAs per SM, 128 registers per thread as in the 512-thread
// shape.  Algorithm 4's column blocks run in this shape: a team of a few CTAs
// per block gets twice as many CTAs, so more of its pivot's dependent loads
// are in flight at once.
#define CSS_GREEDY_NT 256
#define CSS_GREEDY_CTAS_PER_SM 2
#define CSS_GREEDY_SHAPE two_per_sm
#include "greedy.cu"

static_assert(CSS_GREEDY_NT == css::kGreedyThreadsPaired, "the paired shape's thread count");
