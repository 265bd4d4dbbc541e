"""GB300-native divide-and-merge graph-index build (ScaleGANN, arxiv 2605.10135).

The compute path is the C-ABI library ``libann.so`` (hand-written CUDA for
sm_103a); :mod:`paper_2605_10135_gb300.ann` is its thin ctypes binding.
"""
__all__ = ["datagen", "configs"]
