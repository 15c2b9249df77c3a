"""Measurement conventions (no GPU work here).

PAPER_FLOPS_PER_PAIR is the flop count of one P2P interaction in the paper's
convention (Table 1: 70 for Biot-Savart plus 104 for stretching); the
sustained-performance formula of Sec. 4.5 multiplies it by the number of
pair interactions and divides by the wall-clock time.
"""
PAPER_FLOPS_PER_PAIR = 174


def paper_flops(pairs, seconds):
    """flop/s in the Table 1 convention for `pairs` interactions in `seconds`."""
    return PAPER_FLOPS_PER_PAIR * float(pairs) / float(seconds)
