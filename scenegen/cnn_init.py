"""Seeded initial parameters for the elimination proposal network (random
draws only; He-style scaling by fan-in).  Flat order: W1[32][6][3][3] b1[32]
W2..W5 [32][32][3][3] with b2..b5 [32], Wh[32], bh[1]."""
import numpy as np

from .rng import Stream

SHAPES = ([((32, 6, 3, 3), 54), ((32,), 0)] + [((32, 32, 3, 3), 288), ((32,), 0)] * 4
          + [((32,), 32), ((1,), 0)])


def cnn_init(seed, scale=1.0, head_bias=0.0):
    s = Stream(seed, 900)
    parts = []
    for shape, fan_in in SHAPES:
        n = int(np.prod(shape))
        parts.append(s.normal(n) * scale * np.sqrt(2.0 / fan_in) if fan_in else np.zeros(n))
    p = np.concatenate(parts)
    p[-1] = head_bias
    return p.astype(np.float32)
