"""GB300-native Morse-Smale complex 1-skeleton (arXiv:2009.03707): libmsc + its binding.

``import paper_2009_03707_gb300.msc`` loads the CUDA library (built in-tree by
``paper_2009_03707_gb300.build.build()``); there is no CPU fallback.
"""
