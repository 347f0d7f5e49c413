"""GB300-native fixed-step cable-network engine (CoreNEURON's compute path).

The engine is the CUDA library ``libcn.so`` behind the C ABI in
``include/cn.h``; :mod:`paper_1901_10975_gb300.cn` is its ctypes binding and
:mod:`paper_1901_10975_gb300.build` compiles the library in-tree.
"""
