"""GB300-native bottom-up adaptive-sketching H2 construction (sm_103a CUDA).

The compute path lives in the CUDA shared library built from ``csrc/``; this
package only marshals arguments to its C ABI.
"""
