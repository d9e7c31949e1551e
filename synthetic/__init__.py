"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests and the benchmark.

This package draws random numbers and lays them out; it holds none of the codec's arithmetic
(no convolution, quantisation, scale indexing, CDF construction or entropy coding).

* :mod:`synthetic.video`   -- moving-texture RGB uint8 chunks (the paper's 1080p / 720p / 4K test
  resolutions stand in for its UVG, MCL-JCV and HEVC sequences, which are not available).
* :mod:`synthetic.weights` -- random-init network weights, N(0, 2/fan_in), in the flat blob layout
  that both ``ufvc_create`` and the oracle accept.
* :mod:`synthetic.symbols` -- quantised-latent stress symbols round(mu + Laplace(0, b)).
"""
from .video import moving_texture, chunk_frames  # noqa: F401
from .weights import layer_table, draw_weights, ARCHS, mean_layer_table, draw_mean_weights, \
    temporal_layer_table, draw_temporal_weights, \
    dc_layer_table, draw_dc_weights  # noqa: F401
from .symbols import laplace_symbols  # noqa: F401
