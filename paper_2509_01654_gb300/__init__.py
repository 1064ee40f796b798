"""GB300-native all-pairs Needleman-Wunsch scoring of phoneme-coded words.

The compute path is the C-ABI library ``libnw`` (CUDA for sm_103a); the Python
module ``paper_2509_01654_gb300.nw`` marshals arguments into it.  Importing the
package loads nothing; ``nw.load_library()`` loads the built library and
raises if it is missing.
"""
