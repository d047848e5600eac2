"""Rounding-error bound of the BF16 tensor-core backward pass (test helper).

Every operand of a tensor-core product is rounded to BF16, 8 significand
bits, with relative error at most u = 2^-9. A gradient value g is a sum of
products p_r (one per vertex-frame row and path through the network), and
each product's factors come out of a chain of earlier rounded operands. To
first order in u the computed value is sum_r p_r (1 + e_r) with
|e_r| <= k u, k the number of roundings along the longest chain that feeds
a product, so

    |g_bf16 - g| <= k u sum_r |p_r| = k u m,

m being what the oracle's magnitude pass returns (the same reverse pass on
absolute values). Counting the roundings of the deepest chain, which ends in
the grid gradient: dL/do, Wo, dpre3, W3, dpre2, W2, dpre1 and W1[:, :Z] on
the way back (8), the forward activations h1, h2, h3 and the weights that
produced them (5), and o's rounding seen through the Eq. 5-7 Jacobian (1):
14; k = 16 leaves room for the FP32 accumulation of up to millions of rows
(each adds at most ~2^-24 relative per addition level). The bound is applied
per parameter block in the 2-norm:

    ||g_bf16 - g||_2 <= k u ||m||_2.

Where the products of a block cancel (a bias gradient adds one signed term per
row, the coarse grid levels many), ||m|| is much larger than ||g||, and the
bound grows with it: that cancellation is what the per-block tolerance has to
follow. A LeakyReLU whose BF16 pre-activation falls on the other side of zero
than the FP64 one switches its derivative between 1 and the slope; such
flips need a pre-activation within k u of zero relative to its magnitude, are
rare, and are not covered by the first-order argument (they are part of what
the margin between 14 and 16 absorbs).
"""
import numpy as np

U_BF16 = 2.0 ** -9
K_ROUNDINGS = 16


def bf16_block_bound(magnitude):
    """The 2-norm bound k u ||m||_2 of one parameter block."""
    return K_ROUNDINGS * U_BF16 * float(np.linalg.norm(np.asarray(magnitude, np.float64)))
