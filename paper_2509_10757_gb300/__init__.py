"""FastTrack tracking hot path on GB300: stereo matching and search of local
map points as hand-written sm_103a CUDA behind a C ABI (``libfasttrack.so``).

Import is light: the CUDA library is loaded on first use by ``_lib``.
"""
__all__ = ["scenes"]
