"""GB300-native CTrex projection / correction / backprojection library."""
