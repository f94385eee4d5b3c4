"""GB300-native frequency-domain EMRI waveform mode sum (arXiv 2307.12585, Sec. 2.2).

The compute path is the CUDA library ``libemri_fd.so`` built from ``csrc/``;
``api`` is its thin Python binding (argument marshalling only).
"""
